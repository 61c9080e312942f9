"""Right-hand side of the multicomponent reacting Navier-Stokes equations
(Methods, Governing equations; Methods, Numerical method).

Conserved variables U = (rho Y_1 .. rho Y_Ns, rho u, rho v, rho w, E), stored
variable-major [nv, nz, ny, nx].  The RHS is

  dU/dt = - sum_d (Fhat^a_{f+1} - Fhat^a_f) / h_d + sum_d (F^d_{f+1} - F^d_f) / h_d + S,
  S = (omega_1 .. omega_Ns, 0, 0, 0, q_L).

`flags` switches terms off for tests: keys 'inviscid', 'viscous', 'chemistry',
'laser' (all default True); 'scheme' picks the inviscid reconstruction
('weno3z' or 'teno6'); 'splitting' 'component' (default) or 'characteristic'
(oracle.charwise, Cartesian grids); 'nscbc' maps an axis whose bc is 2 to its {side: Side}
(oracle.nscbc; a missing side is an outflow with the defaults).  A grid with
node coordinates (oracle.mapped.MappedGridT) runs the mapped form: face fluxes
through the faces' area vectors, divided by the cell volumes.
"""
from __future__ import annotations

import torch

from . import charwise, chemistry, fluxes, laser as laser_mod, mapped, nscbc, thermo, transport
from .mech import R_U, MechT


def _flag(flags, k):
    return True if flags is None else bool(flags.get(k, True))


def primitives(mech: MechT, U: torch.Tensor, T0: torch.Tensor, maxit: int = 30):
    """Conserved -> primitive state (Methods, Governing equations; EOS)."""
    ns = mech.ns
    rho_s = U[:ns]
    rho = rho_s.sum(0)
    vel = [U[ns + k] / rho for k in range(3)]
    Y = rho_s / rho
    e = U[ns + 3] / rho - 0.5 * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2)
    T, conv, its = thermo.temperature_from_energy(mech, Y, e, T0, maxit=maxit)
    Wbar = thermo.mean_molar_mass(mech, Y)
    p = thermo.pressure(mech, rho, Y, T)
    c = thermo.sound_speed(mech, rho, p, Y, T, Wbar)
    X = Y * Wbar / thermo._bcast(mech.W, T)
    return dict(rho=rho, rho_s=rho_s, vel=vel, Y=Y, e=e, T=T, converged=conv, iterations=its,
                Wbar=Wbar, p=p, c=c, X=X)


def cell_state(mech: MechT, U, T0, maxit: int = 30):
    """Primitives plus transport coefficients of every cell."""
    st = primitives(mech, U, T0, maxit)
    T = st["T"]
    cp_s = thermo.species_cp(mech, T)
    mu_s = transport.species_viscosity(mech, T)
    lam_s = transport.species_conductivity(mech, mu_s, cp_s)
    phi = transport.wilke_phi(mech, mu_s)
    st["mu"] = transport.wilke_mixture(st["X"], mu_s, phi)
    st["lam"] = transport.wilke_mixture(st["X"], lam_s, phi)
    Dij = transport.binary_diffusivity(mech, T, st["p"])
    Ds = transport.mixture_diffusivity(mech, st["X"], Dij)
    st["D"] = Ds
    st["Dc"] = st["rho"] * Ds * thermo._bcast(mech.W, T) / st["Wbar"]
    st["h_s"] = thermo.species_h(mech, T)
    st["cp"] = (st["Y"] * cp_s).sum(0)
    return st


def init_state(mech: MechT, prim: torch.Tensor):
    """Primitive fields (p, T, u, v, w, Y_1..Y_Ns) -> (U, T)."""
    ns = mech.ns
    p, T = prim[0], prim[1]
    vel = [prim[2], prim[3], prim[4]]
    Y = prim[5:5 + ns]
    Wbar = thermo.mean_molar_mass(mech, Y)
    rho = p * Wbar / (R_U * T)
    e = (Y * thermo.species_e(mech, T)).sum(0)
    U = torch.empty((ns + 4,) + T.shape, dtype=torch.float64)
    U[:ns] = rho * Y
    for k in range(3):
        U[ns + k] = rho * vel[k]
    U[ns + 3] = rho * (e + 0.5 * (vel[0] ** 2 + vel[1] ** 2 + vel[2] ** 2))
    return U, T.clone()


def rhs(mech: MechT, grid, U: torch.Tensor, T0: torch.Tensor, t: float = 0.0, las=None,
        flags=None, maxit: int = 30, return_state: bool = False):
    """dU/dt and the temperature of every cell.  Raises if a Newton solve fails."""
    ns = mech.ns
    st = cell_state(mech, U, T0, maxit)
    if not bool(st["converged"].all()):
        raise FloatingPointError("temperature Newton iteration did not converge")
    T = st["T"]
    out = torch.zeros_like(U)
    if _flag(flags, "chemistry"):
        out[:ns] = out[:ns] + chemistry.production_rates(mech, st["rho_s"], T)
    if _flag(flags, "laser") and las is not None:
        out[ns + 3] = out[ns + 3] + laser_mod.laser_source(grid, t, las)

    Up = fluxes.pad(U, grid)
    velp = [fluxes.pad(v, grid) for v in st["vel"]]
    Tp = fluxes.pad(T, grid)
    pp = fluxes.pad(st["p"], grid)
    cp = fluxes.pad(st["c"], grid)
    if _flag(flags, "viscous"):
        Xp = fluxes.pad(st["X"], grid)
        Yp = fluxes.pad(st["Y"], grid)
        Dcp = fluxes.pad(st["Dc"], grid)
        hp = fluxes.pad(st["h_s"], grid)
        mup = fluxes.pad(st["mu"], grid)
        lamp = fluxes.pad(st["lam"], grid)
    scheme = (flags or {}).get("scheme", "weno3z")
    charw = (flags or {}).get("splitting", "component") == "characteristic"
    if getattr(grid, "nodes", None) is not None:
        if charw:
            raise ValueError("characteristic-wise splitting is stated for Cartesian grids only")
        geo = mapped.cached_geometry(grid)
        Vp = fluxes.pad(geo["V"], grid)
        Mp = fluxes.pad(geo["M"], grid)
        for d in range(3):
            if _flag(flags, "inviscid"):
                Fa = mapped.inviscid_flux(Up, velp, pp, cp, Vp, geo["S"][d], grid, d, ns, scheme)
                out = out - mapped.divergence(Fa, grid, d, geo["V"])
                if grid.bc[d] == nscbc.BC_NSCBC:
                    out = nscbc.correct_mapped(mech, grid, geo, st, U, Fa, out, d, (flags or {}).get("nscbc", {}).get(d))
            if _flag(flags, "viscous"):
                Fd = mapped.diffusive_flux(velp, Tp, Xp, Yp, Dcp, hp, mup, lamp, Mp, geo["S"][d], grid, d, ns)
                out = out + mapped.divergence(Fd, grid, d, geo["V"])
        if return_state:
            return out, T, st
        return out, T
    for d in range(3):
        if _flag(flags, "inviscid"):
            if charw:
                Fa = charwise.inviscid_flux(mech, Up, velp, pp, cp, Tp, grid, d, ns, scheme)
            else:
                Fa = fluxes.inviscid_flux(Up, velp, pp, cp, grid, d, ns, scheme)
            out = out - fluxes.divergence(Fa, grid, d)
            if grid.bc[d] == nscbc.BC_NSCBC:
                out = nscbc.correct(mech, grid, st, Fa, out, d, (flags or {}).get("nscbc", {}).get(d))
        if _flag(flags, "viscous"):
            Fd = fluxes.diffusive_flux(velp, Tp, Xp, Yp, Dcp, hp, mup, lamp, grid, d, ns)
            out = out + fluxes.divergence(Fd, grid, d)
    if return_state:
        return out, T, st
    return out, T
