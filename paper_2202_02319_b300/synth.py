"""Seeded synthetic inputs: reaction mechanisms and primitive initial fields.

This module draws the inputs that both the CUDA path and the FP64 oracle consume:
species data (molar masses, NASA-7 coefficient sets, transport parameters),
element-balanced reversible Arrhenius mechanisms, and the primitive fields
(p, T, u, v, w, Y_s) of the synthetic workloads that stand in for the paper's
diffusion-flame (Sec. 4.1) and jet-ignition (Sec. 4.2) cases.

It holds no step of the solver's arithmetic: it never forms conserved
variables, never evaluates a flux, a rate or a temperature solve.  The only
physics used here is what is needed to *design* sensible inputs (the NASA-7
integration constants that place h(298 K) at a drawn formation enthalpy, and
an ideal-gas sound speed used to scale a synthetic velocity field).

Every random number comes from a counter-based Philox stream keyed by
(seed, stream name), so a draw never depends on the order in which other
inputs were generated.
"""
from __future__ import annotations

import zlib
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

R_GAS = 8.314462618      # J/mol/K
P_ATM = 101325.0         # Pa
T_REF = 298.15           # K, reference temperature of formation data

BC_PERIODIC = 0
BC_EXTRAPOLATE = 1
BC_NSCBC = 2


def stream(seed: int, name: str) -> np.random.Generator:
    """Philox generator for the named sub-stream of `seed`."""
    ss = np.random.SeedSequence(entropy=int(seed), spawn_key=(zlib.crc32(name.encode()),))
    return np.random.Generator(np.random.Philox(ss))


# --------------------------------------------------------------------------- mechanism

@dataclass
class Mechanism:
    """Species and reaction data, all in SI units.

    nasa_low / nasa_high: [Ns, 7] NASA-7 coefficient sets (a1..a7) for
    T < T_mid and T >= T_mid.  A: [Nr] pre-exponential factor in
    (m^3/mol)^(n-1)/s with n the reaction order.  nu_f / nu_r: [Nr, Ns]
    reactant / product stoichiometric coefficients.
    """
    names: List[str]
    W: np.ndarray
    elem: np.ndarray
    nasa_low: np.ndarray
    nasa_high: np.ndarray
    T_mid: np.ndarray
    mu_ref: np.ndarray
    mu_exp: np.ndarray
    D_ref: np.ndarray
    A: np.ndarray
    b: np.ndarray
    Theta: np.ndarray
    nu_f: np.ndarray
    nu_r: np.ndarray
    reversible: np.ndarray
    # pressure-dependent reactions (None: every reaction elementary).  rxn_type [Nr]:
    # 0 elementary, 1 third body (rate times [M] = sum_s efficiency_s C_s), 2 Lindemann
    # and 3 Troe fall-off (A, b, Theta the high-pressure limit, A0, b0, Theta0 the
    # low-pressure one in (m^3/mol)^order / s, troe [Nr, 4] = alpha, T***, T*, T**)
    rxn_type: Optional[np.ndarray] = None
    efficiency: Optional[np.ndarray] = None
    A0: Optional[np.ndarray] = None
    b0: Optional[np.ndarray] = None
    Theta0: Optional[np.ndarray] = None
    troe: Optional[np.ndarray] = None

    @property
    def n_species(self) -> int:
        return len(self.names)

    @property
    def n_reactions(self) -> int:
        return int(self.A.shape[0])

    @property
    def n_elements(self) -> int:
        return int(self.elem.shape[1])

    def index(self, name: str) -> int:
        return self.names.index(name)


def _nasa_from_cp_poly(c: np.ndarray, h_f: float, s0: float) -> np.ndarray:
    """NASA-7 set whose cp/R is the quartic `c` (c[k] multiplies T^k), whose
    enthalpy equals h_f [J/mol] and whose entropy equals s0 [J/mol/K] at 298.15 K."""
    T = T_REF
    a = np.zeros(7)
    a[:5] = c
    sens_h = sum(c[k] * T ** (k + 1) / (k + 1) for k in range(5))          # int_0^T cp/R dT
    a[5] = h_f / R_GAS - sens_h
    sens_s = c[0] * np.log(T) + sum(c[k] * T ** k / k for k in range(1, 5))
    a[6] = s0 / R_GAS - sens_s
    return a


def _fit_cp(cp300: float, cp3000: float) -> np.ndarray:
    """Least-squares quartic on [200, 6000] K of cp/R(T) = c0 + c1 (1 - exp(-T/1000))
    anchored at cp/R(300) and cp/R(3000)."""
    e1, e2 = np.exp(-0.3), np.exp(-3.0)
    c1 = (cp3000 - cp300) / (e1 - e2)
    c0 = cp300 - c1 * (1.0 - e1)
    T = np.linspace(200.0, 6000.0, 600)
    y = c0 + c1 * (1.0 - np.exp(-T / 1000.0))
    t = T / 1000.0
    V = np.stack([t ** k for k in range(5)], axis=1)
    coef, *_ = np.linalg.lstsq(V, y, rcond=None)
    return coef / 1000.0 ** np.arange(5)


def _transport(g: np.random.Generator, ns: int):
    mu_ref = g.uniform(1.0e-5, 2.5e-5, ns)
    mu_exp = g.uniform(0.6, 0.8, ns)
    D = np.zeros((ns, ns))
    for i in range(ns):
        for j in range(i + 1, ns):
            D[i, j] = D[j, i] = g.uniform(1.0e-5, 8.0e-5)
    for i in range(ns):
        D[i, i] = g.uniform(1.0e-5, 8.0e-5)      # self-diffusion: never used by the method
    return mu_ref, mu_exp, D


def _arrhenius(g: np.random.Generator, nu_f: np.ndarray, nu_r: np.ndarray, h_f: np.ndarray):
    """A log-uniform in [1e8, 1e13] (CHEMKIN units), b in [-1, 1], Theta in
    [5000, 20000] K.  The drawn Theta is the barrier of the exothermic direction:
    a reaction that is endothermic as written (at 298 K) adds dh/R to it, so that
    the reverse rate k_f / K_c never has a negative activation temperature."""
    nr = nu_f.shape[0]
    A_cgs = 10.0 ** g.uniform(8.0, 13.0, nr)
    b = g.uniform(-1.0, 1.0, nr)
    Theta = g.uniform(5000.0, 20000.0, nr)
    dh = (nu_r - nu_f) @ h_f
    Theta = Theta + np.maximum(dh, 0.0) / R_GAS
    order = nu_f.sum(axis=1)
    A = A_cgs * (1.0e-6) ** (order - 1)            # (cm^3/mol)^(n-1)/s -> (m^3/mol)^(n-1)/s
    return A, b, Theta


def _entropy(g: np.random.Generator, atoms: float) -> float:
    """s(298) in [100, 250] J/mol/K, growing with molecular size so that reaction
    entropies stay in the physical range."""
    return 115.0 + 45.0 * (atoms - 1.0) + g.uniform(-10.0, 10.0)


def mechanism_4sp(seed: int = 0) -> Mechanism:
    """4 species {X2, Y2, XY, X2Y}, 3 reversible reactions, constant per-species cp."""
    names = ["X2", "Y2", "XY", "X2Y"]
    elem = np.array([[2, 0], [0, 2], [1, 1], [2, 1]], dtype=np.float64)
    g = stream(seed, "mech4/elements")
    w_el = np.array([g.uniform(8.0, 9.0), g.uniform(14.0, 16.0)]) * 1.0e-3
    W = elem @ w_el
    g = stream(seed, "mech4/thermo")
    nasa = np.zeros((4, 7))
    hf_all = np.zeros(4)
    kinds = {"X2": "base", "Y2": "base", "XY": "radical", "X2Y": "product"}
    for s, nm in enumerate(names):
        while True:                                 # redraw until gamma_s <= 5/3
            cp = g.uniform(900.0, 1500.0)
            if cp / (cp - R_GAS / W[s]) <= 5.0 / 3.0:
                break
        h_f = {"base": 0.0, "radical": g.uniform(30e3, 250e3),
               "product": g.uniform(-300e3, -100e3)}[kinds[nm]]
        s0 = _entropy(g, elem[s].sum())
        hf_all[s] = h_f
        c = np.zeros(5)
        c[0] = cp * W[s] / R_GAS
        nasa[s] = _nasa_from_cp_poly(c, h_f, s0)
    mu_ref, mu_exp, D = _transport(stream(seed, "mech4/transport"), 4)
    #            X2 Y2 XY X2Y
    nu_f = np.array([[1, 1, 0, 0],     # X2 + Y2   <=> 2 XY
                     [1, 0, 2, 0],     # X2 + 2 XY <=> 2 X2Y
                     [2, 1, 0, 0]])    # 2 X2 + Y2 <=> 2 X2Y
    nu_r = np.array([[0, 0, 2, 0],
                     [0, 0, 0, 2],
                     [0, 0, 0, 2]])
    A, b, Theta = _arrhenius(stream(seed, "mech4/arrhenius"), nu_f, nu_r, hf_all)
    return Mechanism(names, W, elem, nasa.copy(), nasa.copy(), np.full(4, 1000.0),
                     mu_ref, mu_exp, D, A, b, Theta, nu_f, nu_r, np.ones(3, dtype=np.int32))


_SP9 = ["X", "Y", "X2", "Y2", "XY", "X2Y", "XY2", "X2Y2", "Z2"]
_EL9 = np.array([[1, 0, 0], [0, 1, 0], [2, 0, 0], [0, 2, 0], [1, 1, 0],
                 [2, 1, 0], [1, 2, 0], [2, 2, 0], [0, 0, 2]], dtype=np.float64)


def balanced_reactions(elem: np.ndarray, reactive: List[int]):
    """All element-balanced reactions with 1-2 reactant and 1-2 product molecules
    drawn from `reactive`, one orientation per reversible pair."""
    sides = []
    for i, a in enumerate(reactive):
        sides.append((a,))
        for b in reactive[i:]:
            sides.append((a, b))
    out = []
    for i, r in enumerate(sides):
        for p in sides[i + 1:]:
            if set(r) & set(p):
                continue
            if np.array_equal(elem[list(r)].sum(0), elem[list(p)].sum(0)):
                out.append((r, p))
    return out


def mechanism_9sp(seed: int = 0, n_reactions: int = 19) -> Mechanism:
    """9 species {X, Y, X2, Y2, XY, X2Y, XY2, X2Y2, Z2} (Z2 inert), `n_reactions`
    reversible element-balanced reactions, NASA-7 fits of a smooth drawn cp(T)."""
    names = list(_SP9)
    elem = _EL9.copy()
    g = stream(seed, "mech9/elements")
    w_el = np.array([g.uniform(1.0, 2.0), g.uniform(14.0, 16.0), g.uniform(12.0, 14.0)]) * 1.0e-3
    W = elem @ w_el
    g = stream(seed, "mech9/thermo")
    kinds = {"X": "radical", "Y": "radical", "XY": "radical", "X2": "base", "Y2": "base",
             "Z2": "base", "X2Y": "product", "XY2": "product", "X2Y2": "product"}
    nasa = np.zeros((9, 7))
    hf_all = np.zeros(9)
    for s, nm in enumerate(names):
        cp300 = g.uniform(2.5, 4.5)
        cp3000 = cp300 + g.uniform(0.5, 3.0)
        c = _fit_cp(cp300, cp3000)
        h_f = {"base": 0.0, "radical": g.uniform(30e3, 250e3),
               "product": g.uniform(-300e3, -100e3)}[kinds[nm]]
        s0 = _entropy(g, elem[s].sum())
        hf_all[s] = h_f
        nasa[s] = _nasa_from_cp_poly(c, h_f, s0)
    mu_ref, mu_exp, D = _transport(stream(seed, "mech9/transport"), 9)

    cands = balanced_reactions(elem, list(range(8)))
    iX2, iY2, iX2Y = names.index("X2"), names.index("Y2"), names.index("X2Y")

    def orient(rx, want_reactants=None, want_product=None):
        r, p = rx
        if want_reactants is not None and sorted(p) == sorted(want_reactants):
            return (p, r)
        if want_product is not None and want_product in r:
            return (p, r)
        return (r, p)

    g = stream(seed, "mech9/reactions")
    init = [c for c in cands if sorted(c[0]) == sorted((iX2, iY2)) or sorted(c[1]) == sorted((iX2, iY2))]
    chosen = [orient(init[g.integers(len(init))], want_reactants=(iX2, iY2))]
    prod = [c for c in cands if (iX2Y in c[0] or iX2Y in c[1]) and
            sorted(map(sorted, c)) != sorted(map(sorted, chosen[0]))]
    chosen.append(orient(prod[g.integers(len(prod))], want_product=iX2Y))
    taken = {tuple(sorted((tuple(sorted(c[0])), tuple(sorted(c[1]))))) for c in chosen}
    rest = [c for c in cands if tuple(sorted((tuple(sorted(c[0])), tuple(sorted(c[1]))))) not in taken]
    pick = g.permutation(len(rest))[: n_reactions - 2]
    chosen += [rest[k] for k in sorted(pick)]
    nr = len(chosen)
    nu_f = np.zeros((nr, 9), dtype=np.int64)
    nu_r = np.zeros((nr, 9), dtype=np.int64)
    for j, (r, p) in enumerate(chosen):
        for s in r:
            nu_f[j, s] += 1
        for s in p:
            nu_r[j, s] += 1
    A, b, Theta = _arrhenius(stream(seed, "mech9/arrhenius"), nu_f, nu_r, hf_all)
    return Mechanism(names, W, elem, nasa.copy(), nasa.copy(), np.full(9, 1000.0),
                     mu_ref, mu_exp, D, A, b, Theta, nu_f, nu_r, np.ones(nr, dtype=np.int32))


def mechanism_9sp_pressure(seed: int = 0, n_reactions: int = 19) -> Mechanism:
    """mechanism_9sp with pressure-dependent reactions: of the reactions that join
    two molecules into one (or split one into two), the first becomes a third-body
    reaction, the second a Lindemann fall-off and the third a Troe fall-off.
    Efficiencies U[0.5, 3] (the inert Z2 at 1); low-pressure limits with
    P_r = k0 [M] / k_inf of order one at 1 atm and 1000 K."""
    m = mechanism_9sp(seed, n_reactions)
    nr, ns = m.n_reactions, m.n_species
    g = stream(seed, "mech9/pressure")
    rt = np.zeros(nr, dtype=np.int32)
    eff = np.ones((nr, ns))
    A0, b0, Th0 = m.A.copy(), m.b.copy(), m.Theta.copy()
    troe = np.zeros((nr, 4))
    cand = [j for j in range(nr) if sorted((int(m.nu_f[j].sum()), int(m.nu_r[j].sum()))) == [1, 2]]
    for kind, j in zip((1, 2, 3), cand):
        rt[j] = kind
        eff[j] = g.uniform(0.5, 3.0, ns)
        eff[j, m.index("Z2")] = 1.0
        if kind >= 2:
            A0[j] = m.A[j] * g.uniform(0.01, 1.0)
            b0[j] = m.b[j] - g.uniform(0.5, 1.5)
            Th0[j] = m.Theta[j] * g.uniform(0.5, 0.9)
        if kind == 3:
            troe[j] = [g.uniform(0.3, 0.8), g.uniform(100.0, 300.0), g.uniform(1000.0, 3000.0), g.uniform(3000.0, 6000.0)]
    m.rxn_type, m.efficiency, m.A0, m.b0, m.Theta0, m.troe = rt, eff, A0, b0, Th0, troe
    return m


# --------------------------------------------------------------------------- cases

@dataclass
class Grid:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    bc: tuple = (BC_PERIODIC, BC_PERIODIC, BC_PERIODIC)

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz


@dataclass
class Laser:
    """Gaussian energy deposition (Sec. 6.4.1 Eq. for q_L): energy E [J], centre
    (x0, y0, z0) [m], spatial width sigma_r [m], peak time t0 [s], duration sigma_t [s]."""
    E: float = 0.0
    x0: float = 0.0
    y0: float = 0.0
    z0: float = 0.0
    sigma_r: float = 1.0
    t0: float = 0.0
    sigma_t: float = 1.0

    def as_tuple(self):
        return (self.E, self.x0, self.y0, self.z0, self.sigma_r, self.t0, self.sigma_t)


@dataclass
class Case:
    """A workload: mechanism, grid, primitive fields prim[5+Ns, nz, ny, nx] in the
    order (p, T, u, v, w, Y_1..Y_Ns) (a numpy array, or a torch tensor for the
    jet-in-a-box cases), laser and run length."""
    name: str
    mech: Mechanism
    grid: Grid
    prim: np.ndarray
    laser: Laser = field(default_factory=Laser)
    steps: int = 10
    cfl: float = 0.5
    # characteristic boundaries: (axis, side) -> {p_inf, sigma, eta_u, eta_T, eta_t,
    # eta_Y, length, target}; target None (outflow) or [4 + Ns, plane] (u, v, w, T, Y_s)
    # on the boundary plane, plane index t1 + n_t1 t2 over the two other axes
    nscbc: dict = field(default_factory=dict)
    # mapped grids: node (cell corner) coordinates [3, nz + 1, ny + 1, nx + 1], else None
    nodes: Optional[np.ndarray] = None


def _centres(n: int, d: float) -> np.ndarray:
    return (np.arange(n) + 0.5) * d


def _solenoidal(g: np.random.Generator, shape, kmask_fn, spectrum_fn=None):
    """Random divergence-free velocity on a periodic box via FFT: complex Gaussian
    modes, amplitude sqrt(E(k)/(4 pi k^2)) (or 1 inside the mask), projected onto
    the plane normal to k."""
    nz, ny, nx = shape
    kz = np.fft.fftfreq(nz) * nz
    ky = np.fft.fftfreq(ny) * ny
    kx = np.fft.rfftfreq(nx) * nx
    KZ, KY, KX = np.meshgrid(kz, ky, kx, indexing="ij")
    k2 = KX ** 2 + KY ** 2 + KZ ** 2
    k = np.sqrt(k2)
    amp = np.where(kmask_fn(k), 1.0, 0.0)
    if spectrum_fn is not None:
        with np.errstate(divide="ignore", invalid="ignore"):
            amp = amp * np.sqrt(np.where(k > 0, spectrum_fn(k) / (4 * np.pi * np.maximum(k2, 1e-30)), 0.0))
    shp = KX.shape
    a = [(g.standard_normal(shp) + 1j * g.standard_normal(shp)) * amp for _ in range(3)]
    with np.errstate(divide="ignore", invalid="ignore"):
        kd = (KX * a[0] + KY * a[1] + KZ * a[2]) / np.where(k2 > 0, k2, 1.0)
    a = [a[0] - KX * kd, a[1] - KY * kd, a[2] - KZ * kd]
    return [np.fft.irfftn(c, s=shape, axes=(0, 1, 2)) for c in a]


def _cp_mix_R(mech: Mechanism, Y: np.ndarray, T: np.ndarray) -> np.ndarray:
    """Molar-free cp [J/kg/K] of the drawn polynomial fits, used only to scale inputs."""
    a = mech.nasa_low
    cpR = sum(a[:, k][:, None] * T.reshape(1, -1) ** k for k in range(5))    # [Ns, n]
    return (Y.reshape(mech.n_species, -1) * cpR * (R_GAS / mech.W)[:, None]).sum(0).reshape(T.shape)


def _sound_speed(mech: Mechanism, Y: np.ndarray, T: np.ndarray) -> np.ndarray:
    Rm = (Y * (R_GAS / mech.W)[(slice(None),) + (None,) * T.ndim]).sum(0)
    cp = _cp_mix_R(mech, Y, T)
    return np.sqrt(cp / (cp - Rm) * Rm * T)


def case_box32(seed: int = 0) -> Case:
    """32^3 periodic box, 4 species, constant cp: T = 300 K plus a Gaussian hot kernel
    peaking at 1500 K (sigma 4 cells), mass fractions from one Dirichlet(1,1,1,1) draw
    modulated by +-50 % smooth random modes |k| <= 4 (a per-cell draw would be
    grid-scale white noise), random solenoidal Fourier modes |k| <= 4 scaled to
    max |u|/c = 0.3, p = 1 atm."""
    mech = mechanism_4sp(seed)
    n, dx = 32, 1.0e-4
    grid = Grid(n, n, n, dx, dx, dx)
    x = _centres(n, dx)
    Z, Y_, X = np.meshgrid(x, x, x, indexing="ij")
    c = n * dx / 2
    r2 = (X - c) ** 2 + (Y_ - c) ** 2 + (Z - c) ** 2
    T = 300.0 + 1200.0 * np.exp(-r2 / (2 * (4 * dx) ** 2))
    gY = stream(seed, "box32/Y")
    base = gY.dirichlet(np.ones(4))
    w = np.empty((4, n, n, n))
    for s_ in range(4):
        phi = _solenoidal(gY, (n, n, n), lambda k: (k > 0) & (k <= 4.0))[0]
        w[s_] = base[s_] * (1.0 + 0.5 * phi / np.abs(phi).max())
    Yf = w / w.sum(0)
    u = _solenoidal(stream(seed, "box32/u"), (n, n, n), lambda k: (k > 0) & (k <= 4.0))
    umag = np.sqrt(u[0] ** 2 + u[1] ** 2 + u[2] ** 2)
    scale = 0.3 / np.max(umag / _sound_speed(mech, Yf, T))
    prim = np.concatenate([np.full((1, n, n, n), P_ATM), T[None], *(scale * ui[None] for ui in u), Yf])
    return Case("box32_4sp", mech, grid, prim, Laser(), steps=10)


def _air(mech: Mechanism) -> np.ndarray:
    y = np.zeros(mech.n_species)
    y[mech.index("Y2")] = 0.233
    y[mech.index("Z2")] = 0.767
    return y


def _fuel(mech: Mechanism) -> np.ndarray:
    y = np.zeros(mech.n_species)
    y[mech.index("X2")] = 1.0
    return y


def case_mixing_layer(seed: int = 0, n: int = 512) -> Case:
    """2-D mixing layer n x n x 1 (periodic in x, zero-gradient in y): fuel (X2, Y = 1,
    300 K, u = +50 m/s) against air-like oxidiser (Y2/Z2, 1200 K, u = -50 m/s), tanh
    profile 8 cells thick, 1 % white noise on u and v, p = 1 atm."""
    mech = mechanism_9sp(seed)
    dx = 1.0e-4
    grid = Grid(n, n, 1, dx, dx, dx, (BC_PERIODIC, BC_EXTRAPOLATE, BC_PERIODIC))
    y = _centres(n, dx)
    phi = 0.5 * (1.0 + np.tanh((y - n * dx / 2) / (4.0 * dx)))            # 0 fuel -> 1 oxidiser
    phi = np.ascontiguousarray(np.broadcast_to(phi[None, :, None], (1, n, n)))
    g = stream(seed, "mix2d/noise")
    u = 50.0 * (1.0 - 2.0 * phi) + 0.5 * g.standard_normal((1, n, n))
    v = 0.5 * g.standard_normal((1, n, n))
    T = 300.0 + 900.0 * phi
    Yf = (1.0 - phi)[None] * _fuel(mech)[:, None, None, None] + phi[None] * _air(mech)[:, None, None, None]
    prim = np.concatenate([np.full((1, 1, n, n), P_ATM), T[None], u[None], v[None],
                           np.zeros((1, 1, n, n)), Yf])
    return Case(f"mixing_layer_{n}x{n}", mech, grid, prim, Laser(), steps=200)


def case_jet_inflow(seed: int = 0, nx: int = 64, ny: int = 48, nz: int = 1, u_jet: float = 100.0,
                    u_co: float = 5.0, noise: float = 0.01) -> Case:
    """Injection through characteristic boundaries, after the paper's diffusion flame
    (an oxidiser jet from the centre of the left boundary into quiescent fuel, a slow
    fuel co-flow from the rest of that boundary, NSCBC inflow on the left and outflow
    on the right): nx x ny x nz cells of 1e-4 m, x an NSCBC axis, y and z zero-gradient.
    The domain starts as fuel (X2) at 1 atm and 300 K moving at u_co, with white noise
    of rms noise * u_jet on every velocity component (w only in 3-D).  Inflow target: air-like oxidiser in the jet (radius ny / 8
    cells about the plane's centre, tanh edge one cell wide) at u_jet, fuel at u_co
    elsewhere, 300 K; relaxation coefficients eta = 1.  Outflow: p_inf = 1 atm,
    sigma = 0.25."""
    mech = mechanism_9sp(seed)
    dx = 1.0e-4
    bcz = BC_EXTRAPOLATE if nz > 1 else BC_PERIODIC
    grid = Grid(nx, ny, nz, dx, dx, dx, (BC_NSCBC, BC_EXTRAPOLATE, bcz))
    g = stream(seed, f"jetin{nx}x{ny}x{nz}/noise")
    shape = (nz, ny, nx)
    fu, ox = _fuel(mech), _air(mech)
    prim = np.zeros((5 + mech.n_species,) + shape)
    prim[0] = P_ATM
    prim[1] = 300.0
    prim[2] = u_co + noise * u_jet * g.standard_normal(shape)
    prim[3] = noise * u_jet * g.standard_normal(shape)
    if nz > 1:
        prim[4] = noise * u_jet * g.standard_normal(shape)
    prim[5:] = fu[:, None, None, None]
    yc = _centres(ny, dx) - ny * dx / 2
    zc = _centres(nz, dx) - nz * dx / 2 if nz > 1 else np.zeros(1)
    r = np.sqrt(yc[None, :] ** 2 + zc[:, None] ** 2)                        # [nz, ny]
    phi = 0.5 * (1.0 - np.tanh((r - (ny / 8) * dx) / dx))                   # 1 in the jet
    target = np.zeros((4 + mech.n_species, nz, ny))
    target[0] = u_co + (u_jet - u_co) * phi
    target[3] = 300.0
    target[4:] = phi[None] * ox[:, None, None] + (1.0 - phi)[None] * fu[:, None, None]
    sides = {(0, 0): dict(p_inf=P_ATM, target=target.reshape(4 + mech.n_species, nz * ny)),
             (0, 1): dict(p_inf=P_ATM, sigma=0.25, target=None)}
    return Case(f"jet_inflow_{nx}x{ny}x{nz}", mech, grid, prim, Laser(), steps=100, nscbc=sides)


def skewed_nodes(N: int, L: float = 10.0, beta: float = 0.2, dz: Optional[float] = None) -> np.ndarray:
    """The skewed grid of the paper's convergence tests (Solver Performance
    Analysis, Accuracy): the uniform N x N nodes (xi, eta) of [-L/2, L/2]^2 placed at
    x = xi (1 + beta sin(2 pi eta / L)), y = eta (1 + beta sin(2 pi xi / L)), one cell
    deep (z nodes 0 and dz, default L / N).  Shape [3, 2, N + 1, N + 1]."""
    h = L / N
    s_ = -L / 2 + np.arange(N + 1) * h
    E, Xi = np.meshgrid(s_, s_, indexing="ij")
    x = Xi * (1.0 + beta * np.sin(2 * np.pi * E / L))
    y = E * (1.0 + beta * np.sin(2 * np.pi * Xi / L))
    dz = h if dz is None else dz
    return np.stack([np.stack([x, x]), np.stack([y, y]),
                     np.stack([np.zeros_like(x), np.full_like(x, dz)])])


def wavy_nodes(nx: int, ny: int, nz: int, h: float, amp: float = 0.2) -> np.ndarray:
    """A translation-periodic curved grid: the uniform nodes of spacing h moved by
    amp h times products of sines of period (nx, ny, nz) cells in the other two
    indices, so that every cell is curved and sheared and the grid tiles space
    periodically.  Shape [3, nz + 1, ny + 1, nx + 1]."""
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    a, b, c = 2 * np.pi * i / nx, 2 * np.pi * j / ny, 2 * np.pi * k / max(nz, 1)
    X = np.stack([i * h, j * h, k * h]).astype(np.float64)
    X[0] += amp * h * np.sin(b) * (np.cos(c) if nz > 1 else 1.0)
    X[1] += amp * h * np.sin(a) * (np.cos(c) if nz > 1 else 1.0)
    if nz > 1:
        X[2] += amp * h * np.sin(a) * np.sin(b)
    return X


def case_jet_mapped(seed: int = 0, n: int = 64, amp: float = 0.2, device=None) -> Case:
    """The jet in a periodic box (case_jet's fields, n^3 cells) on a curved,
    translation-periodic grid (wavy_nodes, amplitude amp cells): the curvilinear
    workload."""
    c = case_jet(seed, n, device=device)
    c.name = f"jet_mapped_{n}^3"
    c.nodes = wavy_nodes(n, n, n, c.grid.dx, amp)
    return c


def _torch_gen(seed: int, name: str, device):
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(zlib.crc32(f"{int(seed)}/{name}".encode()))
    return g


def _jet_box(mech: Mechanism, seed: int, tag: str, shape, dx: float, r_jet: float,
             turb: bool = True, device=None):
    """Jet-in-a-box primitive fields as a float64 torch tensor [5+Ns, nz, ny, nx] on
    `device` (default CPU): fuel jet along x of radius r_jet (tanh edge, 2 cells),
    air-like oxidiser, p = 1 atm, T = 300 K, plus a von Karman turbulence field
    E(k) ~ k^4 / (1 + (k/k_e)^2)^(17/6), k_e = 1/r_jet, solenoidal, rms 5 m/s per
    component.  Random numbers come from torch's generator on `device`, seeded by
    (seed, tag), so a case is reproducible on the device that generated it."""
    import torch
    dev = torch.device(device if device is not None else "cpu")
    f64 = torch.float64
    nz, ny, nx = shape
    zc = (torch.arange(nz, device=dev, dtype=f64) + 0.5) * dx - nz * dx / 2
    yc = (torch.arange(ny, device=dev, dtype=f64) + 0.5) * dx - ny * dx / 2
    r = torch.sqrt(yc[None, :] ** 2 + zc[:, None] ** 2)
    phi2 = 0.5 * (1.0 - torch.tanh((r - r_jet) / (2.0 * dx)))            # [nz, ny], 1 in the jet
    prim = torch.empty((5 + mech.n_species,) + tuple(shape), dtype=f64, device=dev)
    phi = phi2[:, :, None].expand(shape)
    prim[0].fill_(P_ATM)
    prim[1].fill_(300.0)
    prim[2].copy_(100.0 * phi)
    prim[3].zero_()
    prim[4].zero_()
    fu, ox = _fuel(mech), _air(mech)
    for s_ in range(mech.n_species):
        prim[5 + s_].copy_(phi * float(fu[s_]) + (1.0 - phi) * float(ox[s_]))
    if turb:
        g = _torch_gen(seed, tag + "/turb", dev)
        kz = torch.fft.fftfreq(nz, device=dev, dtype=f64) * nz
        ky = torch.fft.fftfreq(ny, device=dev, dtype=f64) * ny
        kx = torch.fft.rfftfreq(nx, device=dev, dtype=f64) * nx
        KZ, KY, KX = kz[:, None, None], ky[None, :, None], kx[None, None, :]
        k2 = KX ** 2 + KY ** 2 + KZ ** 2
        k = torch.sqrt(k2)
        ke = 1.0 / (r_jet / dx)
        kk = k * (2.0 * np.pi / min(shape))
        spec = kk ** 4 / (1.0 + (kk / ke) ** 2) ** (17.0 / 6.0)
        amp = torch.where(k > 0, torch.sqrt(spec / (4 * np.pi * torch.clamp(k2, min=1e-30))), torch.zeros_like(k))
        cshape = k.shape
        a = [torch.complex(torch.randn(cshape, generator=g, device=dev, dtype=f64),
                           torch.randn(cshape, generator=g, device=dev, dtype=f64)) * amp for _ in range(3)]
        kd = (KX * a[0] + KY * a[1] + KZ * a[2]) / torch.where(k2 > 0, k2, torch.ones_like(k2))
        a = [a[0] - KX * kd, a[1] - KY * kd, a[2] - KZ * kd]
        t = [torch.fft.irfftn(c, s=tuple(shape), dim=(0, 1, 2)) for c in a]
        del a, kd
        rms = torch.sqrt((t[0] ** 2 + t[1] ** 2 + t[2] ** 2).mean() / 3.0)
        for i in range(3):
            prim[2 + i].add_(t[i] * (5.0 / rms))
    return prim


JET_DX = 3.0e-4     # m; places the configs' 5-40 mJ, 3-cell laser kernels at 1000-4500 K


def case_jet(seed: int = 0, n: int = 256, device=None) -> Case:
    """3-D jet in a periodic box n^3: fuel jet (X2) of radius 16 n/256 cells (at
    least 2) along x at 100 m/s into quiescent air-like oxidiser at 1 atm and
    300 K, von Karman turbulence at 5 % of 100 m/s, and a 20 mJ Gaussian laser
    (sigma_r = 3 cells, sigma_t = 10 ns) at a seeded point on the shear layer."""
    mech = mechanism_9sp(seed)
    dx = JET_DX
    r_jet = max(2, (16 * n) // 256) * dx
    grid = Grid(n, n, n, dx, dx, dx)
    prim = _jet_box(mech, seed, f"jet{n}", (n, n, n), dx, r_jet, device=device)
    g = stream(seed, f"jet{n}/laser")
    th = g.uniform(0.0, 2.0 * np.pi)
    las = Laser(E=20e-3, x0=g.uniform(0.25, 0.75) * n * dx,
                y0=n * dx / 2 + r_jet * np.cos(th), z0=n * dx / 2 + r_jet * np.sin(th),
                sigma_r=3.0 * dx, t0=1.0e-6, sigma_t=10e-9)
    return Case(f"jet_{n}^3", mech, grid, prim, las, steps=100)


def ensemble_members(seed: int = 0, n_members: int = 64, lo: int = 48, hi: int = 96,
                     t0_max: float = 50e-6, device=None) -> List[Case]:
    """Batched-ensemble workload: each member a jet-in-a-box with every axis drawn
    from U{lo..hi}, jet radius min(ny, nz)/8 cells, laser energy U[5, 40] mJ at a
    point on the shear layer, deposition time U[0, t0_max]."""
    mech = mechanism_9sp(seed)
    dx = JET_DX
    g = stream(seed, "ensemble/members")
    out = []
    for m in range(n_members):
        nx, ny, nz = (int(v) for v in g.integers(lo, hi + 1, size=3))
        r_jet = max(2, min(ny, nz) // 8) * dx
        prim = _jet_box(mech, seed, f"ensemble/{m}", (nz, ny, nx), dx, r_jet, device=device)
        th = g.uniform(0.0, 2.0 * np.pi)
        las = Laser(E=g.uniform(5e-3, 40e-3), x0=g.uniform(0.25, 0.75) * nx * dx,
                    y0=ny * dx / 2 + r_jet * np.cos(th), z0=nz * dx / 2 + r_jet * np.sin(th),
                    sigma_r=3.0 * dx, t0=g.uniform(0.0, t0_max), sigma_t=10e-9)
        out.append(Case(f"member{m}_{nx}x{ny}x{nz}", mech, Grid(nx, ny, nz, dx, dx, dx), prim, las, steps=10))
    return out


def adjoint_members(seed: int = 0, n_members: int = 16, n: int = 64, t0: float = 0.0) -> List[Case]:
    """Sensitivity workload: members sharing the n^3 jet-in-a-box state of
    case_jet(seed, n), each with its own laser (energy U[5, 40] mJ at a point on
    the shear layer, sigma_r = 3 cells, sigma_t = 10 ns, deposition time t0)."""
    base = case_jet(seed, n)
    g = stream(seed, f"adjoint/{n}/members")
    dx = base.grid.dx
    r_jet = max(2, (16 * n) // 256) * dx
    out = []
    for m in range(n_members):
        th = g.uniform(0.0, 2.0 * np.pi)
        las = Laser(E=g.uniform(5e-3, 40e-3), x0=g.uniform(0.25, 0.75) * n * dx,
                    y0=n * dx / 2 + r_jet * np.cos(th), z0=n * dx / 2 + r_jet * np.sin(th),
                    sigma_r=3.0 * dx, t0=t0, sigma_t=10e-9)
        out.append(Case(f"adjoint_member{m}_{n}^3", base.mech, base.grid, base.prim, las, steps=200))
    return out
