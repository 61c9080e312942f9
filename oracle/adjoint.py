"""Discrete gradients of the oracle by reverse-mode automatic differentiation of
the oracle's own functions (a library primitive serving as the transpose).

Objective, restating the ignition measure: J = sum_n dt sum_k b_k H(U^(k)) over
fixed-dt SSP-RK3 steps, stage inputs U^(0) = U^n, U^(1), U^(2) at times t, t+dt,
t+dt/2 with b = (1/6, 1/6, 2/3); H = sum over cells of -sum_s h_s omega_s dV.
"""
from __future__ import annotations

import torch

from . import chemistry, rhs as rhs_mod, thermo


def heat_release(mech, grid, U, T0):
    st = rhs_mod.primitives(mech, U, T0)
    w = chemistry.production_rates(mech, st["rho_s"], st["T"])
    hrr = chemistry.heat_release_rate(mech, w, st["T"])
    return hrr.sum() * grid.dx * grid.dy * grid.dz, st["T"]


def step_objective(mech, grid, U, T, t, dt, las, flags=None):
    """One step in the same stage order as the CUDA path; returns (U_next, T, dJ)."""
    b = (1.0 / 6.0, 1.0 / 6.0, 2.0 / 3.0)
    H0, _ = heat_release(mech, grid, U, T)
    R0, T = rhs_mod.rhs(mech, grid, U, T, t, las, flags)
    U1 = U + dt * R0
    H1, _ = heat_release(mech, grid, U1, T)
    R1, T = rhs_mod.rhs(mech, grid, U1, T, t + dt, las, flags)
    U2 = 0.75 * U + 0.25 * (U1 + dt * R1)
    H2, _ = heat_release(mech, grid, U2, T)
    R2, T = rhs_mod.rhs(mech, grid, U2, T, t + 0.5 * dt, las, flags)
    Un = U / 3.0 + (2.0 / 3.0) * (U2 + dt * R2)
    return Un, T.detach(), dt * (b[0] * H0 + b[1] * H1 + b[2] * H2)


def objective(mech, grid, U0, T0, t0, dt, nsteps, las, lnA=None, flags=None):
    """J for parameters given as tensors (laser tuple entries, lnA) so that
    torch.autograd.grad gives dJ/dp."""
    m = mech.with_A(torch.exp(lnA)) if lnA is not None else mech
    U, T = U0, T0
    J = torch.zeros((), dtype=torch.float64)
    for k in range(nsteps):
        U, T, dJ = step_objective(m, grid, U, T, t0 + k * dt, dt, las, flags)
        J = J + dJ
    return J
