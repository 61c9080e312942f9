"""Pins of the oracle's characteristic boundaries (Application examples: the
diffusion flame and the combustor use NSCBC inflow and outflow boundaries, after
Poinsot & Lele 1992 and Okong'o & Bellan 2002), each against something outside
the boundary code: the Euler flux and the conserved-variable map of the oracle's
pinned thermodynamics (by finite differences), the LODI relations for the
primitive rates at a boundary, the structure of the correction (interior cells
untouched, a uniform state at its targets at rest), and the behaviour the
method exists for (an acoustic pulse leaves the domain, the pressure relaxes
towards p_inf)."""
import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import fluxes, nscbc, rhs, rk, thermo
from oracle.mech import GridT, R_U
from tests.helpers import mech_t, random_prim, tensor

NO_SRC = {"chemistry": False, "laser": False, "viscous": False}


@pytest.fixture(scope="module")
def mech():
    return mech_t(synth.mechanism_4sp(0))


def _U_of_V(mt, rho, vel, p, Y):
    """Conserved variables of the primitive state (rho, u, v, w, p, Y) through the
    oracle's EOS and internal energy."""
    Wbar = thermo.mean_molar_mass(mt, Y)
    T = p * Wbar / (rho * R_U)
    prim = torch.cat([p[None], T[None], vel[0][None], vel[1][None], vel[2][None], Y])
    U, _ = rhs.init_state(mt, prim)
    return U


def _random_states(mt, n, seed):
    g = np.random.default_rng(seed)
    ns = mt.ns
    shape = (1, 1, n)
    p = tensor(g.uniform(5e4, 3e5, shape))
    T = tensor(g.uniform(300.0, 2400.0, shape))
    vel = [tensor(g.uniform(-200.0, 200.0, shape)) for _ in range(3)]
    Y = tensor(g.dirichlet(np.ones(ns), size=shape).transpose(3, 0, 1, 2))
    Wbar = thermo.mean_molar_mass(mt, Y)
    rho = p * Wbar / (R_U * T)
    c = thermo.sound_speed(mt, rho, p, Y, T, Wbar)
    return g, rho, vel, p, Y, T, c


def _zero_sum(g, ns, shape, scale):
    r = g.standard_normal((ns,) + shape)
    r -= r.mean(0, keepdims=True)
    return tensor(scale * r)


@pytest.mark.parametrize("d", [0, 1, 2])
def test_conserved_form_maps_the_primitive_rates(mech, d):
    """-P(V) d equals dU/dt of the primitive rates (drho, dp, du_k, dY)/dt =
    -(d1, d2, d_k, dY), by central differences of the conserved map U(V): pins
    the momentum and the multicomponent energy closure."""
    g, rho, vel, p, Y, T, c = _random_states(mech, 24, 1 + d)
    shape = rho.shape
    ns = mech.ns
    rdot = tensor(g.standard_normal(shape)) * 0.01 * rho
    pdot = tensor(g.standard_normal(shape)) * 0.01 * p
    udot = [tensor(g.standard_normal(shape)) * 10.0 for _ in range(3)]
    Ydot = _zero_sum(g, ns, shape, 0.01)
    t1, t2 = [a for a in range(3) if a != d]
    d1, d2, dY = -rdot, -pdot, -Ydot
    d3, d4, d5 = -udot[d], -udot[t1], -udot[t2]
    # amplitudes with these d: L5 + L1 = 2 d2, L5 - L1 = 2 rho c d3, L2 = c^2 d1 - d2
    L1 = d2 - rho * c * d3
    L5 = d2 + rho * c * d3
    L2 = c * c * d1 - d2
    got = nscbc.characteristic_term(mech, rho, vel, p, Y, T, c, d, (L1, L2, d4, d5, L5, dY))
    eps = 1e-6
    Up = _U_of_V(mech, rho + eps * rdot, [v + eps * w for v, w in zip(vel, udot)], p + eps * pdot, Y + eps * Ydot)
    Um = _U_of_V(mech, rho - eps * rdot, [v - eps * w for v, w in zip(vel, udot)], p - eps * pdot, Y - eps * Ydot)
    want = (Up - Um) / (2 * eps)
    scale = want.abs().amax(dim=(1, 2, 3), keepdim=True) + 1e-300
    assert float(((got - want).abs() / scale).max()) < 1e-7


@pytest.mark.parametrize("d", [0, 1, 2])
def test_unreplaced_waves_give_the_euler_flux_derivative(mech, d):
    """With every amplitude kept, -P d(L) is -dF/dn of the Euler flux along d for
    the primitive gradient dV/dn (central differences of F(U(V))): pins the wave
    decomposition, the frozen sound speed and the conserved form together."""
    g, rho, vel, p, Y, T, c = _random_states(mech, 24, 11 + d)
    shape = rho.shape
    ns = mech.ns
    drho = tensor(g.standard_normal(shape)) * 50.0 * rho
    dp = tensor(g.standard_normal(shape)) * 50.0 * p
    dvel = [tensor(g.standard_normal(shape)) * 5e4 for _ in range(3)]
    dY = _zero_sum(g, ns, shape, 50.0)
    t1, t2 = [a for a in range(3) if a != d]
    L = nscbc.amplitudes(rho, vel[d], vel[t1], vel[t2], p, Y, c, drho, dvel[d], dvel[t1], dvel[t2], dp, dY)
    got = nscbc.characteristic_term(mech, rho, vel, p, Y, T, c, d, L)

    def F(s):
        r, pv, Yv = rho + s * drho, p + s * dp, Y + s * dY
        v = [a + s * b for a, b in zip(vel, dvel)]
        return fluxes.euler_flux(_U_of_V(mech, r, v, pv, Yv), v, pv, d, ns)
    eps = 1e-9
    want = -(F(eps) - F(-eps)) / (2 * eps)
    scale = want.abs().amax(dim=(1, 2, 3), keepdim=True) + 1e-300
    assert float(((got - want).abs() / scale).max()) < 1e-6


def _uniform(mt, n3, p, T, vel, Y):
    nz, ny, nx = n3
    prim = torch.empty((5 + mt.ns, nz, ny, nx), dtype=torch.float64)
    prim[0], prim[1] = p, T
    for k in range(3):
        prim[2 + k] = vel[k]
    prim[5:] = tensor(Y)[:, None, None, None]
    return rhs.init_state(mt, prim)


def _prim_rates(mt, U, T, R, eps):
    """Central-difference rates of (rho, u, v, w, p, T, Y) along dU/dt = R."""
    def prim(V):
        st = rhs.primitives(mt, V, T)
        return [st["rho"], *st["vel"], st["p"], st["T"], *st["Y"]]
    a, b = prim(U + eps * R), prim(U - eps * R)
    return [(x - y) / (2 * eps) for x, y in zip(a, b)]


def test_outflow_relaxes_pressure_at_the_lodi_rate(mech):
    """Uniform subsonic flow along x at p != p_inf, outflow sides at both ends:
    at the boundary cells dp/dt = -K (p - p_inf) / 2 and du/dt = -+K (p - p_inf) /
    (2 rho c) (low / high end), K = sigma c (1 - M^2) / ell; the interior is at rest."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, pinf, u0, T0 = 1.02e5, 1.0e5, 40.0, 600.0
    g = GridT(8, 1, 1, 1e-3, 1e-3, 1e-3, (2, 0, 0))
    U, T = _uniform(mech, (1, 1, 8), p0, T0, (u0, 0.0, 0.0), Y)
    sides = {0: nscbc.Side(p_inf=pinf, sigma=0.3), 1: nscbc.Side(p_inf=pinf, sigma=0.3)}
    R, _ = rhs.rhs(mech, g, U, T, flags=dict(NO_SRC, nscbc={0: sides}))
    assert float(R[..., 1:7].abs().max()) == 0.0
    st = rhs.primitives(mech, U, T)
    rho, c = float(st["rho"].flatten()[0]), float(st["c"].flatten()[0])
    K = 0.3 * c * (1.0 - (u0 / c) ** 2) / (8 * 1e-3)
    rates = _prim_rates(mech, U, T, R, 1e-9)
    for i, sgn in ((0, -1.0), (7, 1.0)):
        dp = float(rates[4][0, 0, i])
        du = float(rates[1][0, 0, i])
        assert dp == pytest.approx(-K * (p0 - pinf) / 2, rel=1e-6)
        assert du == pytest.approx(sgn * K * (p0 - pinf) / (2 * rho * c), rel=1e-6)
        assert float(rates[2][0, 0, i]) == pytest.approx(0.0, abs=1e-6)
        for s in range(4):
            assert float(rates[6 + s][0, 0, i]) == pytest.approx(0.0, abs=1e-9)


def test_inflow_relaxes_velocity_temperature_and_composition(mech):
    """Uniform flow entering at the low end with a target (u, v, w, T, Y): the
    boundary cell's primitive rates are the LODI ones of the replaced amplitudes
    (drho/dt = -(L2 + L5/2)/c^2, dp/dt = -L5/2, du/dt = -L5/(2 rho c),
    dv/dt = -L3, dw/dt = -L4, dY/dt = -LY)."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    Yt = np.array([0.25, 0.25, 0.2, 0.3])
    p0, u0, T0 = 1.0e5, 30.0, 500.0
    tgt = (36.0, 4.0, -3.0, 560.0)
    nx, dx = 8, 1e-3
    g = GridT(nx, 2, 1, dx, dx, dx, (2, 0, 0))
    U, T = _uniform(mech, (1, 2, nx), p0, T0, (u0, 0.0, 0.0), Y)
    target = torch.empty((4 + 4, 1, 2), dtype=torch.float64)
    for k, v in enumerate(tgt):
        target[k] = v
    target[4:] = tensor(Yt)[:, None, None]
    spec = nscbc.Side(p_inf=p0, eta_u=0.7, eta_T=0.9, eta_t=0.5, eta_Y=0.8, target=target)
    R, _ = rhs.rhs(mech, g, U, T, flags=dict(NO_SRC, nscbc={0: {0: spec, 1: nscbc.Side(p_inf=p0)}}))
    st = rhs.primitives(mech, U, T)
    rho, c = float(st["rho"].flatten()[0]), float(st["c"].flatten()[0])
    Wbar = float(st["Wbar"].flatten()[0])
    ell, F = nx * dx, 1.0 - (u0 / c) ** 2
    L5 = 0.7 * rho * c * c * F * (u0 - tgt[0]) / ell
    L2 = -0.9 * rho * c * (R_U / Wbar) * (T0 - tgt[3]) / ell
    L3 = 0.5 * c / ell * (0.0 - tgt[1])
    L4 = 0.5 * c / ell * (0.0 - tgt[2])
    LY = 0.8 * c / ell * (Y - Yt)
    rates = _prim_rates(mech, U, T, R, 1e-9)
    at = lambda k: float(rates[k][0, 0, 0])  # noqa: E731
    assert at(0) == pytest.approx(-(L2 + 0.5 * L5) / c ** 2, rel=1e-6)
    assert at(4) == pytest.approx(-0.5 * L5, rel=1e-6)
    assert at(1) == pytest.approx(-L5 / (2 * rho * c), rel=1e-6)
    assert at(2) == pytest.approx(-L3, rel=1e-6)
    assert at(3) == pytest.approx(-L4, rel=1e-6)
    for s in range(4):
        assert at(6 + s) == pytest.approx(-LY[s], rel=1e-6)


def test_inflow_temperature_relaxes_at_eta_c_over_gamma_ell(mech):
    """With velocity and composition at their targets only the entropy wave is
    replaced, and T relaxes at dT/dt = -eta_T c (T - T_t) / (gamma ell) (the
    frozen gamma of the mixture)."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, u0, T0, Tt = 1.0e5, 30.0, 500.0, 540.0
    nx, dx = 8, 1e-3
    g = GridT(nx, 1, 1, dx, dx, dx, (2, 0, 0))
    U, T = _uniform(mech, (1, 1, nx), p0, T0, (u0, 0.0, 0.0), Y)
    target = torch.empty((8, 1, 1), dtype=torch.float64)
    target[0], target[1], target[2], target[3] = u0, 0.0, 0.0, Tt
    target[4:] = tensor(Y)[:, None, None]
    spec = nscbc.Side(p_inf=p0, eta_T=0.9, target=target)
    R, _ = rhs.rhs(mech, g, U, T, flags=dict(NO_SRC, nscbc={0: {0: spec, 1: nscbc.Side(p_inf=p0)}}))
    st = rhs.primitives(mech, U, T)
    c, rho = float(st["c"].flatten()[0]), float(st["rho"].flatten()[0])
    gamma = rho * c * c / p0
    rates = _prim_rates(mech, U, T, R, 1e-9)
    assert float(rates[5][0, 0, 0]) == pytest.approx(-0.9 * c * (T0 - Tt) / (gamma * nx * dx), rel=1e-6)
    assert float(rates[4][0, 0, 0]) == pytest.approx(0.0, abs=1e-6 * p0)


def test_uniform_state_at_its_targets_is_at_rest(mech):
    """p = p_inf at the outflow and the inflow target equal to the state: every
    cell's RHS vanishes (viscous terms on; chemistry off)."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, u0, T0 = 1.0e5, 25.0, 450.0
    nx, ny = 8, 3
    g = GridT(nx, ny, 1, 1e-3, 1e-3, 1e-3, (2, 0, 0))
    U, T = _uniform(mech, (1, ny, nx), p0, T0, (u0, 0.0, 0.0), Y)
    target = torch.empty((8, 1, ny), dtype=torch.float64)
    target[0], target[1], target[2], target[3] = u0, 0.0, 0.0, T0
    target[4:] = tensor(Y)[:, None, None]
    flags = {"chemistry": False, "laser": False,
             "nscbc": {0: {0: nscbc.Side(p_inf=p0, target=target), 1: nscbc.Side(p_inf=p0)}}}
    R, _ = rhs.rhs(mech, g, U, T, flags=flags)
    st = rhs.primitives(mech, U, T)
    rho, c = float(st["rho"].max()), float(st["c"].max())
    E = float(U[-1].abs().max())
    scale = torch.tensor([rho] * 4 + [rho * c] * 3 + [E], dtype=torch.float64)[:, None, None, None] * c / 1e-3
    assert float((R.abs() / scale).max()) < 1e-14


def test_interior_cells_match_the_extrapolated_scheme(mech):
    """The correction touches the first and last layer of the NSCBC axis only:
    every other cell's RHS is bitwise that of zero-gradient ghost cells."""
    m = synth.mechanism_4sp(0)
    prim = tensor(random_prim(m, (4, 5, 7), seed=3, smooth=True))
    U, T = rhs.init_state(mech, prim)
    flags = {"laser": False}
    for d in range(3):
        bc_x = [1, 1, 0]
        bc_x[d] = 2
        bc_e = [1, 1, 0]
        bc_e[d] = 1
        gx = GridT(7, 5, 4, 1e-3, 1.2e-3, 0.9e-3, tuple(bc_x))
        ge = GridT(7, 5, 4, 1e-3, 1.2e-3, 0.9e-3, tuple(bc_e))
        Rx, _ = rhs.rhs(mech, gx, U, T, flags=flags)
        Re, _ = rhs.rhs(mech, ge, U, T, flags=flags)
        ax = 4 + fluxes.AX[d]
        n = (7, 5, 4)[d]
        inner = lambda f: f.narrow(ax, 1, n - 2)  # noqa: E731
        assert torch.equal(inner(Rx), inner(Re))
        for b in (0, n - 1):
            assert not torch.equal(Rx.narrow(ax, b, 1), Re.narrow(ax, b, 1))


def _acoustic_pulse(mt, nx, dx, A, x0, w):
    """Right-running linear acoustic pulse on a gas at rest (p' = rho c u' = c^2 rho')."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, T0 = 1.0e5, 300.0
    U0, Tb = _uniform(mt, (1, 1, nx), p0, T0, (0.0, 0.0, 0.0), Y)
    st = rhs.primitives(mt, U0, Tb)
    rho0, c0 = float(st["rho"].flatten()[0]), float(st["c"].flatten()[0])
    x = (torch.arange(nx, dtype=torch.float64) + 0.5) * dx
    pp = A * torch.exp(-((x - x0) / w) ** 2)
    rho = rho0 + pp / c0 ** 2
    p = p0 + pp
    u = pp / (rho0 * c0)
    Wbar = thermo.mean_molar_mass(mt, tensor(Y)[:, None])[0]
    Tf = p * Wbar / (rho * R_U)
    prim = torch.empty((9, 1, 1, nx), dtype=torch.float64)
    prim[0, 0, 0], prim[1, 0, 0], prim[2, 0, 0] = p, Tf, u
    prim[3], prim[4] = 0.0, 0.0
    prim[5:] = tensor(Y)[:, None, None, None]
    U, T = rhs.init_state(mt, prim)
    return U, T, p0, c0


def _run(mt, g, U, T, flags, t_end, cfl=0.5):
    t = 0.0
    while t < t_end:
        U, T, dt = rk.rk_step(mt, g, U, T, t, 0.0, None, cfl, flags)
        t += dt
    return U, T


def test_acoustic_pulse_leaves_through_the_outflow(mech):
    """A right-running pulse of amplitude A crosses the high end of a sigma = 0
    outflow: what stays in the domain once it has left is below 1% of A."""
    nx, dx, A = 100, 1e-4, 50.0
    U, T, p0, c0 = _acoustic_pulse(mech, nx, dx, A, 60 * dx, 5 * dx)
    g = GridT(nx, 1, 1, dx, dx, dx, (2, 0, 0))
    sides = {0: nscbc.Side(p_inf=p0, sigma=0.0), 1: nscbc.Side(p_inf=p0, sigma=0.0)}
    U, T = _run(mech, g, U, T, dict(NO_SRC, nscbc={0: sides}), 70 * dx / c0)
    p = rhs.primitives(mech, U, T)["p"]
    assert float((p - p0).abs().max()) < 0.01 * A


def test_outflow_pressure_relaxes_towards_p_inf(mech):
    """A gas at rest at p_0 != p_inf between two outflow ends (sigma = 0.5) moves
    its mean pressure towards p_inf over a few acoustic times, which zero-gradient
    ghost cells (no p_inf anywhere) do not."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    nx, dx, p0, pinf = 32, 2e-4, 1.01e5, 1.0e5
    U, T = _uniform(mech, (1, 1, nx), p0, 300.0, (0.0, 0.0, 0.0), Y)
    c0 = float(rhs.primitives(mech, U, T)["c"].flatten()[0])
    g = GridT(nx, 1, 1, dx, dx, dx, (2, 0, 0))
    sides = {0: nscbc.Side(p_inf=pinf, sigma=0.5), 1: nscbc.Side(p_inf=pinf, sigma=0.5)}
    t_end = 4 * nx * dx / c0
    Un, Tn = _run(mech, g, U, T, dict(NO_SRC, nscbc={0: sides}), t_end)
    dev = float((rhs.primitives(mech, Un, Tn)["p"] - pinf).mean())
    assert 0.0 <= dev < 0.5 * (p0 - pinf)
    ge = GridT(nx, 1, 1, dx, dx, dx, (1, 0, 0))
    Ue, Te = _run(mech, ge, U, T, NO_SRC, t_end)
    assert float((rhs.primitives(mech, Ue, Te)["p"] - p0).abs().max()) < 1e-6 * p0


@pytest.mark.parametrize("side", [0, 1])
def test_inflow_velocity_relaxes_towards_its_target_at_either_end(mech, side):
    """Flow entering through either end (u_n > 0 at the low end, < 0 at the high
    end) with a velocity target: du_n/dt = -eta_u c (1 - M^2)(u_n - u_n,t) / (2 ell)
    at the boundary cell, towards the target from either side."""
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, T0, nx, dx = 1.0e5, 500.0, 8, 1e-3
    u0 = 30.0 if side == 0 else -30.0
    ut = u0 + 7.0
    g = GridT(nx, 1, 1, dx, dx, dx, (2, 0, 0))
    U, T = _uniform(mech, (1, 1, nx), p0, T0, (u0, 0.0, 0.0), Y)
    target = torch.empty((8, 1, 1), dtype=torch.float64)
    target[0], target[1], target[2], target[3] = ut, 0.0, 0.0, T0
    target[4:] = tensor(Y)[:, None, None]
    sides = {side: nscbc.Side(p_inf=p0, eta_u=0.6, target=target), 1 - side: nscbc.Side(p_inf=p0)}
    R, _ = rhs.rhs(mech, g, U, T, flags=dict(NO_SRC, nscbc={0: sides}))
    c = float(rhs.primitives(mech, U, T)["c"].flatten()[0])
    rates = _prim_rates(mech, U, T, R, 1e-9)
    b = 0 if side == 0 else nx - 1
    want = -0.6 * c * (1.0 - (u0 / c) ** 2) * (u0 - ut) / (2 * nx * dx)
    assert float(rates[1][0, 0, b]) == pytest.approx(want, rel=1e-6)


def _quadratic_state(mt, nx, dx, u_mean):
    """Primitive fields quadratic in x (rho, u, p, Y), v = w = 0."""
    ell = nx * dx
    xi = ((torch.arange(nx, dtype=torch.float64) + 0.5) * dx) / ell

    def q(a0, a1, a2):
        return a0 * (1.0 + a1 * xi + a2 * xi * xi)
    rho = q(1.1, 0.2, -0.15)
    u = q(u_mean, -0.1, 0.08)
    p = q(1.2e5, 0.15, 0.1)
    Yr = torch.stack([q(0.1, 0.3, 0.2), q(0.2, -0.2, 0.1), q(0.3, 0.1, -0.1)])
    Y = torch.cat([Yr, (1.0 - Yr.sum(0))[None]])
    return rho, u, p, Y, xi, ell


@pytest.mark.parametrize("direction", [1.0, -1.0])
def test_supersonic_outflow_gives_the_exact_flux_derivative(mech, direction):
    """Supersonic flow along +x or -x (every wave outgoing at the downstream end,
    incoming at the upstream end), inviscid terms only, primitives quadratic in x:
    the downstream cell's RHS is -dF/dx at its centre exactly (one-sided
    second-order differences are exact for quadratics; the scheme's term is
    replaced, not added); the upstream cell, an outflow side with every wave
    incoming and 1 - M^2 < 0, holds its state (RHS 0)."""
    nx, dx = 10, 1e-3
    u_mean = 900.0 * direction
    rho, u, p, Y, xi, ell = _quadratic_state(mech, nx, dx, u_mean)
    zero = torch.zeros_like(rho)
    U = _U_of_V(mech, rho[None, None], [u[None, None], zero[None, None], zero[None, None]], p[None, None], Y[:, None, None])
    Wbar = thermo.mean_molar_mass(mech, Y)
    T = (p * Wbar / (rho * R_U))[None, None]
    c = float(rhs.primitives(mech, U, T)["c"].max())
    assert float(u.abs().min()) > 1.2 * c
    g = GridT(nx, 1, 1, dx, dx, dx, (2, 0, 0))
    R, _ = rhs.rhs(mech, g, U, T, flags=dict(NO_SRC, nscbc={0: {0: nscbc.Side(), 1: nscbc.Side()}}))

    def F_at(x):
        s = x / ell
        r = 1.1 * (1.0 + 0.2 * s - 0.15 * s * s)
        uu = u_mean * (1.0 - 0.1 * s + 0.08 * s * s)
        pp = 1.2e5 * (1.0 + 0.15 * s + 0.1 * s * s)
        yr = [0.1 * (1.0 + 0.3 * s + 0.2 * s * s), 0.2 * (1.0 - 0.2 * s + 0.1 * s * s), 0.3 * (1.0 + 0.1 * s - 0.1 * s * s)]
        Yv = tensor(yr + [1.0 - sum(yr)])[:, None, None, None]
        one = lambda v: tensor([v])[None, None]  # noqa: E731
        Uv = _U_of_V(mech, one(r), [one(uu), one(0.0), one(0.0)], one(pp), Yv)
        return fluxes.euler_flux(Uv, [one(uu), one(0.0), one(0.0)], one(pp), 0, 4)[:, 0, 0, 0]
    down, up = (nx - 1, 0) if direction > 0 else (0, nx - 1)
    xb = (down + 0.5) * dx
    h = 1e-4 * dx
    want = -(F_at(xb + h) - F_at(xb - h)) / (2 * h)
    got = R[:, 0, 0, down]
    scale = want.abs().max()
    assert float(((got - want).abs() / scale).max()) < 1e-7
    assert float((R[:, 0, 0, up].abs() / scale).max()) < 1e-13


def _mapped_nodes_uniform(nx, ny, nz, dx, dy, dz):
    i = torch.arange(nx + 1, dtype=torch.float64) * dx
    j = torch.arange(ny + 1, dtype=torch.float64) * dy
    k = torch.arange(nz + 1, dtype=torch.float64) * dz
    Z, Yy, X = torch.meshgrid(k, j, i, indexing="ij")
    return torch.stack([X, Yy, Z])


def test_mapped_uniform_nodes_reproduce_the_cartesian_boundaries(mech):
    """Characteristic boundaries on a uniform grid given by its nodes (the mapped
    form: normal from the area vectors, d/dn from |S| / V) give the Cartesian RHS,
    with an inflow target on one end and a relaxing outflow on the other."""
    from oracle import mapped
    m = synth.mechanism_4sp(0)
    nz, ny, nx = 3, 4, 9
    dx, dy, dz = 1.1e-4, 0.9e-4, 1.3e-4
    prim = tensor(random_prim(m, (nz, ny, nx), 8, smooth=True))
    U, T = rhs.init_state(mech, prim)
    target = torch.empty((8, nz, ny), dtype=torch.float64)
    target[0], target[1], target[2], target[3] = 30.0, 5.0, -4.0, 900.0
    target[4:] = tensor(np.array([0.2, 0.3, 0.1, 0.4]))[:, None, None]
    sides = {0: nscbc.Side(p_inf=1.0e5, eta_u=0.7, eta_T=0.9, eta_t=0.5, eta_Y=0.8, target=target),
             1: nscbc.Side(p_inf=1.01e5, sigma=0.3)}
    flags = {"laser": False, "nscbc": {0: sides}}
    gc = GridT(nx, ny, nz, dx, dy, dz, (2, 0, 1))
    gm = mapped.MappedGridT(nx, ny, nz, _mapped_nodes_uniform(nx, ny, nz, dx, dy, dz), (2, 0, 1))
    rc, _ = rhs.rhs(mech, gc, U, T, flags=flags)
    rm, _ = rhs.rhs(mech, gm, U, T, flags=flags)
    num = (rm - rc).reshape(rc.shape[0], -1).abs().amax(1)
    den = rc.reshape(rc.shape[0], -1).abs().amax(1)
    assert float((num / den).max()) < 1e-12


def test_mapped_boundaries_on_a_rotated_grid_match_the_one_dimensional_ones(mech):
    """A uniform grid rotated by 30 degrees, characteristic ends on its first axis,
    data varying along that axis only and the velocity along it: the RHS is the
    one-dimensional Cartesian RHS with the momentum rotated."""
    from oracle import mapped
    m = synth.mechanism_4sp(0)
    nx, ny, h = 16, 3, 1e-4
    prim1 = tensor(random_prim(m, (1, 1, nx), 9, smooth=True))
    prim1[3] = 0.0
    prim1[4] = 0.0
    th = np.radians(30.0)
    cs, sn = float(np.cos(th)), float(np.sin(th))
    X = _mapped_nodes_uniform(nx, ny, 1, h, h, h)
    Xr = X.clone()
    Xr[0] = cs * X[0] - sn * X[1]
    Xr[1] = sn * X[0] + cs * X[1]
    prim2 = prim1.expand(prim1.shape[0], 1, ny, nx).clone()
    prim2[2] = cs * prim1[2]
    prim2[3] = sn * prim1[2]
    U1, T1 = rhs.init_state(mech, prim1)
    U2, T2 = rhs.init_state(mech, prim2)
    s1 = {0: nscbc.Side(p_inf=1.0e5, sigma=0.4), 1: nscbc.Side(p_inf=1.02e5, sigma=0.2)}
    fl = dict(NO_SRC, viscous=True, nscbc={0: s1})
    R1, _ = rhs.rhs(mech, GridT(nx, 1, 1, h, h, h, (2, 0, 0)), U1, T1, flags=fl)
    R2, _ = rhs.rhs(mech, mapped.MappedGridT(nx, ny, 1, Xr, (2, 0, 0)), U2, T2, flags=fl)
    want = R1.expand(R1.shape[0], 1, ny, nx).clone()
    want[4] = cs * R1[4]
    want[5] = sn * R1[4]
    scale = R1.reshape(R1.shape[0], -1).abs().amax(1)
    scale[5] = scale[4]
    scale[6] = scale[4]
    err = (R2 - want).reshape(R2.shape[0], -1).abs().amax(1) / scale
    assert float(err.max()) < 1e-10


def test_mapped_uniform_state_at_its_targets_is_at_rest(mech):
    """A uniform flow on the paper's skewed grid with a characteristic inflow at its
    targets and an outflow at p_inf on the first axis: the RHS vanishes to rounding."""
    from oracle import mapped
    N = 12
    nodes = tensor(synth.skewed_nodes(N, L=N * 1e-4))
    Y = np.array([0.1, 0.2, 0.3, 0.4])
    p0, u0, v0, T0 = 1.0e5, 25.0, 7.0, 450.0
    U, T = _uniform(mech, (1, N, N), p0, T0, (u0, v0, 0.0), Y)
    target = torch.empty((8, 1, N), dtype=torch.float64)
    target[0], target[1], target[2], target[3] = u0, v0, 0.0, T0
    target[4:] = tensor(Y)[:, None, None]
    flags = {"chemistry": False, "laser": False,
             "nscbc": {0: {0: nscbc.Side(p_inf=p0, target=target), 1: nscbc.Side(p_inf=p0)}}}
    R, _ = rhs.rhs(mech, mapped.MappedGridT(N, N, 1, nodes, (2, 0, 0)), U, T, flags=flags)
    st = rhs.primitives(mech, U, T)
    rho, c = float(st["rho"].max()), float(st["c"].max())
    E = float(U[-1].abs().max())
    scale = torch.tensor([rho] * 4 + [rho * c] * 3 + [E], dtype=torch.float64)[:, None, None, None] * c / 1e-4
    assert float((R.abs() / scale).max()) < 1e-12
