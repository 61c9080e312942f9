"""Minimum ignition energy by bisection over ensemble members (Application
examples: the ignition studies sort runs that differ in laser energy into
ignited and failed ones and bracket the threshold).  TEST INFRASTRUCTURE: the
oracle's own statement of the search, run member by member on the oracle's
RHS, against which the batched GPU driver is checked.

Readings (the paper states the criteria in words):
  * a member has ignited when its peak temperature at the end of the window is
    at least T_fail = 600 K (below it the paper calls the run a failure) and its
    total heat release rate sum_cells -sum_s h_s omega_s dV at the end exceeds
    the value at the middle of the window and is positive (the heat release
    grows);
  * each round probes `members` energies evenly spaced strictly inside the
    bracket (lo, hi): E_k = lo + (k + 1)(hi - lo)/(members + 1);
  * the new upper end is the smallest ignited energy of the round (else hi), the
    new lower end the largest failed energy below that upper end (else lo).
"""
from __future__ import annotations

import torch

from . import rk, rhs as rhs_mod
from .adjoint import heat_release


def member_window(mech, grid, prim, las, nsteps: int, dt: float, flags=None):
    """Runs one member over the window; returns (peak T at the end, total HRR at
    the middle, total HRR at the end).  flags as for oracle.rhs.rhs (for example the
    case's characteristic ends)."""
    U, T = rhs_mod.init_state(mech, prim)
    half = nsteps // 2
    t = 0.0
    for _ in range(half):
        U, T, _ = rk.rk_step(mech, grid, U, T, t, dt, las, flags=flags)
        t += dt
    h_mid, T = heat_release(mech, grid, U, T)
    for _ in range(nsteps - half):
        U, T, _ = rk.rk_step(mech, grid, U, T, t, dt, las, flags=flags)
        t += dt
    h_end, T = heat_release(mech, grid, U, T)
    return float(T.max()), float(h_mid), float(h_end)


def is_ignited(peak_T: float, h_mid: float, h_end: float, T_fail: float = 600.0) -> bool:
    return peak_T >= T_fail and h_end > 0.0 and h_end > h_mid


def bisect(outcome_of, lo: float, hi: float, members: int, rounds: int):
    """outcome_of(list of energies) -> list of bools (ignited).  Returns the final
    bracket and the probes of every round."""
    history = []
    for _ in range(rounds):
        probes = [lo + (k + 1) * (hi - lo) / (members + 1) for k in range(members)]
        res = outcome_of(probes)
        up = hi
        for e, ok in zip(probes, res):
            if ok and e < up:
                up = e
        down = lo
        for e, ok in zip(probes, res):
            if not ok and e < up and e > down:
                down = e
        lo, hi = down, up
        history.append((probes, res, (lo, hi)))
    return (lo, hi), history


def minimum_ignition_energy(mech, grid, prim, las_template, E_lo: float, E_hi: float, members: int,
                            rounds: int, nsteps: int, dt: float, T_fail: float = 600.0, flags=None):
    """The oracle's bisection: every probe is one member run on the oracle."""
    def outcome_of(energies):
        out = []
        for E in energies:
            las = (E,) + tuple(las_template[1:])
            out.append(is_ignited(*member_window(mech, grid, prim, las, nsteps, dt, flags), T_fail=T_fail))
        return out
    return bisect(outcome_of, E_lo, E_hi, members, rounds)
