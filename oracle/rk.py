"""SSP-RK3 time integration and the time-step rule.

The paper integrates in time with the third-order strong-stability-preserving
Runge-Kutta method of Gottlieb, Shu and Tadmor (Methods, Numerical method).
Shu-Osher form, stage times t, t + dt, t + dt/2:
  U1   = Un + dt L(Un, t)
  U2   = 3/4 Un + 1/4 (U1 + dt L(U1, t + dt))
  Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2, t + dt/2))

The paper runs its accuracy tests at a fixed dt (Methods, Solver Performance
Analysis, Accuracy).  Reading for production steps, with maxima over cells and
only axes with more than one cell:
  dt = min( CFL / max sum_d (|u_d| + c) / h_d,
            0.25 h_min^2 / max(mu/rho, lambda/(rho cp), max_s D_s),   (viscous on)
            0.2 / max_s |d omega_s / d rho_s|,                          (chemistry on)
            laser clamp )                                               (laser on)
laser clamp: while t + dt reaches the window [t0 - 6 sigma_t, t0 + 6 sigma_t]
and t < t0 + 6 sigma_t, dt <= max(sigma_t / 4, t0 - 6 sigma_t - t).
The temperature array carries the Newton warm start: after a step it holds the
temperature of the last stage's input state.
"""
from __future__ import annotations

import torch

from . import chemistry, mapped, rhs as rhs_mod
from .rhs import _flag


def ssp_rk3(L, U, t: float, dt: float):
    """Generic SSP-RK3 step for dU/dt = L(U, t)."""
    U1 = U + dt * L(U, t)
    U2 = 0.75 * U + 0.25 * (U1 + dt * L(U1, t + dt))
    return U / 3.0 + (2.0 / 3.0) * (U2 + dt * L(U2, t + 0.5 * dt))


def rate_limits(mech, grid, U, T0, flags=None):
    """Per-grid maxima (acoustic rate, diffusive coefficient, chemical rate).  On a
    mapped grid the acoustic rate is sum_e (|u . grad xi_e| + c |grad xi_e|) per cell
    and the diffusive entry is max over cells of the coefficient times
    max_e |grad xi_e|^2 (so the limit is 0.25 / that)."""
    st = rhs_mod.cell_state(mech, U, T0)
    nu = st["mu"] / st["rho"]
    alpha = st["lam"] / (st["rho"] * st["cp"])
    dmax = torch.maximum(torch.maximum(nu, alpha), st["D"].max(0).values)
    ch = chemistry.chemical_rate(mech, st["rho_s"], st["T"])
    if getattr(grid, "nodes", None) is not None:
        ac, g2 = mapped.rate_limits(grid, st)
        return float(ac.max()), float((dmax * g2).max()), float(ch.max())
    ac = torch.zeros_like(st["T"])
    for d in range(3):
        if grid.n[d] > 1:
            ac = ac + (st["vel"][d].abs() + st["c"]) / grid.h[d]
    return float(ac.max()), float(dmax.max()), float(ch.max())


def time_step(mech, grid, U, T0, t: float, las, cfl: float, flags=None) -> float:
    ac, dmax, ch = rate_limits(mech, grid, U, T0, flags)
    dt = cfl / ac if ac > 0.0 else 1.0e300
    active = [grid.h[d] for d in range(3) if grid.n[d] > 1]
    if getattr(grid, "nodes", None) is not None:
        if _flag(flags, "viscous") and active and dmax > 0.0:
            dt = min(dt, 0.25 / dmax)
    elif _flag(flags, "viscous") and active and dmax > 0.0:
        hmin = min(active)
        dt = min(dt, 0.25 * hmin * hmin / dmax)
    if _flag(flags, "chemistry") and ch > 0.0:
        dt = min(dt, 0.2 / ch)
    if _flag(flags, "laser") and las is not None:
        t0, st_ = float(las[5]), float(las[6])
        lo, hi = t0 - 6.0 * st_, t0 + 6.0 * st_
        if t + dt > lo and t < hi:
            dt = min(dt, max(0.25 * st_, lo - t))
    return dt


def rk_step(mech, grid, U, T, t: float, dt: float = 0.0, las=None, cfl: float = 0.5, flags=None):
    """One SSP-RK3 step; dt <= 0 selects the time-step rule.  Returns (U, T, dt)."""
    if dt <= 0.0:
        dt = time_step(mech, grid, U, T, t, las, cfl, flags)
    Tc = [T]

    def L(V, tt):
        out, Tn = rhs_mod.rhs(mech, grid, V, Tc[0], tt, las, flags)
        Tc[0] = Tn
        return out
    Un = ssp_rk3(L, U, t, dt)
    return Un, Tc[0], dt
