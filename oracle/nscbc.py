"""Navier-Stokes characteristic boundary conditions for reacting flows
(Application examples: the diffusion flame's left and right boundaries and the
model combustor's injector inlet and nozzle outlet are NSCBC boundaries, after
Poinsot & Lele, J. Comput. Phys. 101 (1992), with the multicomponent reacting
extension of Okong'o & Bellan, J. Comput. Phys. 176 (2002)).  TEST
INFRASTRUCTURE: the oracle's statement of the boundary treatment.

The paper names the method and its sources but prints no formula; this module
states one reading of it, written out from the characteristic analysis of the
Euler equations in the primitive variables V = (rho, u_n, u_t1, u_t2, p, Y_s)
along the boundary normal n (t1, t2 the other two axes in increasing order):

  * Along an NSCBC axis the interior scheme runs with zero-gradient ghost cells
    (so its viscous, conduction and diffusion fluxes through the boundary face
    are those of a zero normal gradient).  In the first and the last cell layer
    the scheme's inviscid normal term -(Fhat_{f+1} - Fhat_f) / h is replaced by
    the characteristic form -P(V) d, everything else of the cell's RHS (the other
    axes, the diffusive terms, chemistry, laser) is kept.
  * Normal derivatives dV/dn at a boundary cell: one-sided second-order
    differences over the boundary cell and its two inward neighbours,
    (-3 V_0 + 4 V_1 - V_2) / (2h) at the low end, (3 V_{n-1} - 4 V_{n-2} + V_{n-3}) / (2h)
    at the high end (the axis needs n >= 3).
  * Wave amplitudes, c the frozen sound speed (the characteristic speeds of a
    mixture with frozen composition are those of a single gas with that c):
      L1 = (u_n - c)(dp/dn - rho c du_n/dn)      L5 = (u_n + c)(dp/dn + rho c du_n/dn)
      L2 = u_n (c^2 drho/dn - dp/dn)             L3 = u_n du_t1/dn,  L4 = u_n du_t2/dn
      LY_s = u_n dY_s/dn.
  * A wave is incoming where its speed (u_n - c, u_n, u_n + c) points into the
    domain: positive at the low end, negative at the high end.  Incoming
    amplitudes are replaced, outgoing ones kept.  With ell the domain length
    along n (n h unless given), M = |u_n| / c and F = max(1 - M^2, 0):
      outflow side: acoustic K (p - p_inf), K = sigma c F / ell (partially
        non-reflecting pressure relaxation); entropy, shear and species 0.
      inflow side (target u, T, Y on the boundary plane): acoustic
        s eta_u rho c^2 F (u_n - u_n,t) / ell with s = +1 at the low end and -1 at
        the high end; entropy -eta_T rho c Rbar (T - T_t) / ell; shear
        eta_t (c / ell)(u_t - u_t,t); species eta_Y (c / ell)(Y_s - Y_s,t).
    Each relaxes its variable towards the target at a rate of order c / ell.
  * d1 = (L2 + (L5 + L1) / 2) / c^2, d2 = (L5 + L1) / 2, d3 = (L5 - L1) / (2 rho c),
    d4 = L3, d5 = L4, dY_s = LY_s are the rates -drho/dt, -dp/dt, -du_n/dt,
    -du_t1/dt, -du_t2/dt, -dY_s/dt of the normal inviscid term.
  * The conserved form (the reacting extension): with e_s = h_s - R T / W_s,
    gamma = rho c^2 / p and Wbar the mean molar mass,
      -P d [rho Y_s] = -(Y_s d1 + rho dY_s)
      -P d [rho u_k] = -(u_k d1 + rho d_k),   d_n = d3, d_t1 = d4, d_t2 = d5
      -P d [E]       = -(|u|^2 d1 / 2 + rho sum_k u_k d_k) + sum_s e_s (-P d [rho Y_s])
                       + p / (gamma - 1) (d1 / rho - d2 / p + Wbar sum_s dY_s / W_s),
    the last term rho c_v dT/dt from T = p / (rho Rbar) (for one species with
    constant c_p it is the textbook -d2 / (gamma - 1) with the rest cancelling).
  * Written for a boundary normal n: u_n = u . n, the shear amplitude is the vector
    u_n d(u - u_n n)/dn and the velocity rate d_n n + (that vector).  On a Cartesian
    grid n is the axis and d/dn = (1/h) d/d(index).  On a mapped grid (oracle.mapped)
    n is the boundary cell's mean area vector of the axis, S = (S_low + S_high) / 2,
    normalised, d/dn = (|S| / V) d/d(index) (the frozen-metric form of the
    characteristic analysis along the computational axis), ell defaults to the number
    of cells over that factor, the inflow target's normal and tangential parts are
    taken against n, and the scheme's term removed is its face-flux difference over V;
    the metric part of the normal term, -(S_high - S_low) . F(U_b) / V with F the
    cell's own Euler flux, is kept (a uniform flow then stays at rest).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch

from . import fluxes, thermo
from .mech import R_U

BC_NSCBC = 2


@dataclass
class Side:
    """One end of an NSCBC axis.  target None: outflow; else inflow with target
    [4 + Ns, *plane] = (u, v, w, T, Y_1 .. Y_Ns) on the boundary plane (the grid's
    (nz, ny, nx) shape without the normal axis)."""
    p_inf: float = 101325.0
    sigma: float = 0.25
    eta_u: float = 1.0
    eta_T: float = 1.0
    eta_t: float = 1.0
    eta_Y: float = 1.0
    length: float = 0.0
    target: Optional[torch.Tensor] = None


def _layer(f: torch.Tensor, d: int, i: int) -> torch.Tensor:
    """Cells with index i along axis d (the trailing three axes are z, y, x)."""
    return f.select(f.dim() + fluxes.AX[d], i)


def _ddn(f: torch.Tensor, d: int, side: int, n: int, h: float) -> torch.Tensor:
    """One-sided second-order normal derivative at the boundary layer."""
    if side == 0:
        return (-3.0 * _layer(f, d, 0) + 4.0 * _layer(f, d, 1) - _layer(f, d, 2)) / (2.0 * h)
    return (3.0 * _layer(f, d, n - 1) - 4.0 * _layer(f, d, n - 2) + _layer(f, d, n - 3)) / (2.0 * h)


def amplitudes(rho, un, ut1, ut2, p, Y, c, drho, dun, dut1, dut2, dp, dY):
    """(L1, L2, L3, L4, L5, LY) from the state and its normal derivatives."""
    L1 = (un - c) * (dp - rho * c * dun)
    L5 = (un + c) * (dp + rho * c * dun)
    L2 = un * (c * c * drho - dp)
    L3 = un * dut1
    L4 = un * dut2
    LY = un[None] * dY
    return L1, L2, L3, L4, L5, LY


def characteristic_term_n(mech, rho, vel, p, Y, T, c, nvec, L1, L2, Lt, L5, LY):
    """-P(V) d as conserved rates [nv, ...] for the boundary normal nvec (a unit
    vector per cell, [3, ...]); Lt is the tangential shear amplitude as a vector
    ([3, ...], normal to nvec): d_u = d_n nvec + Lt is the velocity rate vector."""
    ns = mech.ns
    d1 = (L2 + 0.5 * (L5 + L1)) / (c * c)
    d2 = 0.5 * (L5 + L1)
    dn = (L5 - L1) / (2.0 * rho * c)
    du = [dn * nvec[k] + Lt[k] for k in range(3)]
    dY = LY
    out = torch.empty((ns + 4,) + rho.shape, dtype=torch.float64)
    out[:ns] = -(Y * d1[None] + rho[None] * dY)
    for k in range(3):
        out[ns + k] = -(vel[k] * d1 + rho * du[k])
    ke = 0.5 * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    gamma = rho * c * c / p
    Wbar = thermo.mean_molar_mass(mech, Y)
    e_s = thermo.species_e(mech, T)
    W = thermo._bcast(mech.W, T)
    dT_term = p / (gamma - 1.0) * (d1 / rho - d2 / p + Wbar * (dY / W).sum(0))
    out[ns + 3] = (-(ke * d1 + rho * (vel[0] * du[0] + vel[1] * du[1] + vel[2] * du[2]))
                   + (e_s * out[:ns]).sum(0) + dT_term)
    return out


def _axis_vector(d, like):
    e = [torch.zeros_like(like) for _ in range(3)]
    e[d] = torch.ones_like(like)
    return torch.stack(e)


def characteristic_term(mech, rho, vel, p, Y, T, c, d: int, L):
    """-P(V) d for the Cartesian normal e_d, L = (L1, L2, L3, L4, L5, LY) with L3, L4
    the shear amplitudes along the other two axes in increasing order."""
    L1, L2, L3, L4, L5, LY = L
    t1, t2 = [a for a in range(3) if a != d]
    Lt = [torch.zeros_like(rho) for _ in range(3)]
    Lt[t1] = L3
    Lt[t2] = L4
    return characteristic_term_n(mech, rho, vel, p, Y, T, c, _axis_vector(d, rho), L1, L2, torch.stack(Lt), L5, LY)


def _dxi(f: torch.Tensor, d: int, side: int, n: int) -> torch.Tensor:
    """One-sided second-order index-space derivative at the boundary layer."""
    if side == 0:
        return 0.5 * (-3.0 * _layer(f, d, 0) + 4.0 * _layer(f, d, 1) - _layer(f, d, 2))
    return 0.5 * (3.0 * _layer(f, d, n - 1) - 4.0 * _layer(f, d, n - 2) + _layer(f, d, n - 3))


def boundary_amplitudes_n(mech, st, d: int, side: int, n_d: int, spec: Side, nvec, kappa):
    """Amplitudes at one boundary layer for the unit normal nvec ([3, layer]) with
    d/dn = kappa d/dxi (kappa = 1/h on a Cartesian grid, |S| / V on a mapped one);
    incoming ones replaced.  Returns (L1, L2, Lt, L5, LY) and the layer state."""
    b = 0 if side == 0 else n_d - 1
    rho, p, c, T = (_layer(st[k], d, b) for k in ("rho", "p", "c", "T"))
    vel = [_layer(v, d, b) for v in st["vel"]]
    Y = _layer(st["Y"], d, b)
    un = nvec[0] * vel[0] + nvec[1] * vel[1] + nvec[2] * vel[2]
    drho = kappa * _dxi(st["rho"], d, side, n_d)
    dp = kappa * _dxi(st["p"], d, side, n_d)
    du = [kappa * _dxi(v, d, side, n_d) for v in st["vel"]]
    dY = kappa[None] * _dxi(st["Y"], d, side, n_d)
    dun = nvec[0] * du[0] + nvec[1] * du[1] + nvec[2] * du[2]
    L1 = (un - c) * (dp - rho * c * dun)
    L5 = (un + c) * (dp + rho * c * dun)
    L2 = un * (c * c * drho - dp)
    Lt = torch.stack([un * (du[k] - dun * nvec[k]) for k in range(3)])
    LY = un[None] * dY

    ell = spec.length if spec.length > 0.0 else n_d / kappa
    F = torch.clamp(1.0 - (un / c) ** 2, min=0.0)

    def incoming(lam):
        return lam > 0.0 if side == 0 else lam < 0.0

    if spec.target is None:
        ac = spec.sigma * c * F / ell * (p - spec.p_inf)
        ent = torch.zeros_like(rho)
        sh = torch.zeros_like(Lt)
        spc = torch.zeros_like(Y)
    else:
        tg = spec.target
        utn = nvec[0] * tg[0] + nvec[1] * tg[1] + nvec[2] * tg[2]
        sgn = 1.0 if side == 0 else -1.0
        ac = sgn * spec.eta_u * rho * c * c * F * (un - utn) / ell
        Rbar = R_U / thermo.mean_molar_mass(mech, Y)
        ent = -spec.eta_T * rho * c * Rbar * (T - tg[3]) / ell
        sh = torch.stack([spec.eta_t * c / ell * ((vel[k] - un * nvec[k]) - (tg[k] - utn * nvec[k])) for k in range(3)])
        spc = spec.eta_Y * (c / ell)[None] * (Y - tg[4:])
    L1 = torch.where(incoming(un - c), ac, L1)
    L5 = torch.where(incoming(un + c), ac, L5)
    inc = incoming(un)
    L2 = torch.where(inc, ent, L2)
    Lt = torch.where(inc[None], sh, Lt)
    LY = torch.where(inc[None], spc, LY)
    return (L1, L2, Lt, L5, LY), (rho, vel, p, Y, T, c)


def _metric_flux(U, vel, p, dS, ns):
    """dS . (F, G, H) of the state U (dS a vector per cell, [3, ...])."""
    theta = dS[0] * vel[0] + dS[1] * vel[1] + dS[2] * vel[2]
    F = theta[None] * U
    for k in range(3):
        F[ns + k] = F[ns + k] + p * dS[k]
    F[ns + 3] = F[ns + 3] + p * theta
    return F


def _correct(mech, st, U, Fa, out, d, n_d, sides, geom):
    """geom(side, b) -> (nvec, kappa, V, dS) of the boundary layer: V divides the
    scheme's face-flux difference, dS = S_high - S_low is the change of the area
    vector across the cell, whose part -dS . F(U_b) / V of the normal term (the
    metric's variation, which the faces of the other axes balance for a uniform flow)
    is kept beside the characteristic term; it vanishes on a Cartesian grid."""
    ax = out.dim() + fluxes.AX[d]
    out = out.clone()
    ns = mech.ns
    for side in (0, 1):
        spec = sides.get(side, Side()) if sides else Side()
        b = 0 if side == 0 else n_d - 1
        nvec, kappa, V, dS = geom(side, b)
        scheme = -(Fa.narrow(ax, b + 1, 1) - Fa.narrow(ax, b, 1)).squeeze(ax) / V
        (L1, L2, Lt, L5, LY), (rho, vel, p, Y, T, c) = boundary_amplitudes_n(mech, st, d, side, n_d, spec, nvec, kappa)
        char = characteristic_term_n(mech, rho, vel, p, Y, T, c, nvec, L1, L2, Lt, L5, LY)
        if dS is not None:
            char = char - _metric_flux(_layer(U, d, b), vel, p, dS, ns) / V
        lay = out.narrow(ax, b, 1).squeeze(ax)
        lay += char - scheme
    return out


def correct(mech, grid, st, Fa: torch.Tensor, out: torch.Tensor, d: int, sides) -> torch.Tensor:
    """Replaces the inviscid normal term of the two boundary layers of axis d.
    Fa: the scheme's inviscid face fluxes along d (faces 0..n); sides: dict
    side -> Side (0 low, 1 high); a missing side is an outflow with the defaults."""
    n, h = grid.n[d], grid.h[d]

    def geom(side, b):
        like = _layer(st["rho"], d, b)
        return _axis_vector(d, like), torch.full_like(like, 1.0 / h), h, None
    return _correct(mech, st, None, Fa, out, d, n, sides, geom)


def correct_mapped(mech, grid, geo, st, U, Fa, out, d, sides):
    """The same on a mapped grid: the boundary normal is the cell's mean area vector
    of axis d, S = (S_low + S_high) / 2, n = S / |S|, d/dn = (|S| / V) d/dxi, the
    scheme's term divides by the cell volume, and the metric part -(S_high - S_low) .
    F(U_b) / V of the normal term stays."""
    n = grid.n[d]
    Sd = geo["S"][d]
    ax = Sd.dim() + fluxes.AX[d]

    def geom(side, b):
        Slo = Sd.narrow(ax, b, 1).squeeze(ax)
        Shi = Sd.narrow(ax, b + 1, 1).squeeze(ax)
        S = 0.5 * (Slo + Shi)
        Sm = torch.sqrt(S[0] ** 2 + S[1] ** 2 + S[2] ** 2)
        V = _layer(geo["V"], d, b)
        return S / Sm[None], Sm / V, V, Shi - Slo
    return _correct(mech, st, U, Fa, out, d, n, sides, geom)
