"""Minimum ignition energy by bisection over batched ensembles (the paper's
ensemble question, Application examples: Ignition of a diffusion flame and of
a model rocket combustor, where members differing in laser energy are sorted
into ignited and failed runs and the threshold is bracketed).

Each round runs `members` copies of one flow state in one batched ensemble, the
copies differing only in laser energy, spread evenly inside the current bracket
[E_lo, E_hi].  After the run window a member counts as ignited when its peak
temperature is at least T_fail (the paper's failure criterion is a peak
temperature below 600 K) and its total heat release rate grew over the second
half of the window (the paper's ignition criterion is growth of the heat
release); otherwise it failed.  The new bracket is [the largest failed energy
below the smallest ignited one, the smallest ignited energy], so each round
narrows the bracket by a factor of up to members + 1.  Responses need not be
monotone in energy: the bracket follows the lowest transition seen.

All arithmetic runs in the CUDA library (run_ensemble, rf_diagnostics); this
module only schedules the rounds and reads the two diagnostics per member.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Tuple

import torch

from . import native as nv


def ignited(max_T_end: float, hrr_mid: float, hrr_end: float, T_fail: float = 600.0) -> bool:
    """The ignition test of one member after its window."""
    return max_T_end >= T_fail and hrr_end > 0.0 and hrr_end > hrr_mid


def next_bracket(energies, outcomes, lo: float, hi: float) -> Tuple[float, float]:
    """Bracket after one round: the smallest ignited energy above, the largest
    failed energy below it (the old ends where a round has none)."""
    ign = [e for e, ok in zip(energies, outcomes) if ok]
    new_hi = min(ign) if ign else hi
    below = [e for e, ok in zip(energies, outcomes) if not ok and e < new_hi]
    new_lo = max(below) if below else lo
    return new_lo, new_hi


def probe_energies(lo: float, hi: float, members: int) -> List[float]:
    return [lo + (hi - lo) * (k + 1) / (members + 1) for k in range(members)]


@dataclass
class Round:
    energies: List[float]
    ignited: List[bool]
    max_T: List[float]
    hrr_mid: List[float]
    hrr_end: List[float]
    bracket: Tuple[float, float]


@dataclass
class Result:
    bracket: Tuple[float, float]
    rounds: List[Round] = field(default_factory=list)
    member_steps: int = 0


class EnsembleIgnition:
    """Members of one case (mechanism, grid, primitive state, laser template)
    whose laser energies the rounds set; contexts and states are allocated once."""

    def __init__(self, case, members: int, nsteps: int, dt: float, precision: int = nv.RF_MIXED,
                 mode: int = nv.ENS_GRAPH, T_fail: float = 600.0, device="cuda"):
        self.case = case
        self.members = int(members)
        self.nsteps = int(nsteps)
        self.dt = float(dt)
        self.mode = mode
        self.T_fail = float(T_fail)
        self.dev = torch.device(device)
        ns, n = case.mech.n_species, case.grid.ncells
        self.prim = torch.as_tensor(case.prim, dtype=torch.float64).reshape(5 + ns, n).to(self.dev)
        self.mech = nv.init_mechanism(case.mech)
        self.ctxs = [nv.create_ctx(self.mech, case.grid, precision) for _ in range(self.members)]
        # characteristic ends of the case (inflow targets shared by the members)
        self.targets = {}
        for (axis, side), spec in getattr(case, "nscbc", {}).items():
            kw = {k: v for k, v in spec.items() if k != "target"}
            tg = spec.get("target")
            if tg is not None:
                tg = torch.as_tensor(tg, dtype=torch.float64).to(self.dev).contiguous()
                self.targets[(axis, side)] = tg
            for ctx in self.ctxs:
                nv.set_nscbc(ctx, axis, side, target=tg, **kw)
        self.Us = [torch.empty((ns + 4, n), dtype=torch.float64, device=self.dev) for _ in range(self.members)]
        self.Ts = [torch.empty(n, dtype=torch.float64, device=self.dev) for _ in range(self.members)]

    def run(self, energies):
        """Runs one round; returns per member (max T, HRR mid, HRR end)."""
        assert len(energies) == self.members
        base = self.case.laser.as_tuple()
        lasers = [(float(E),) + tuple(base[1:]) for E in energies]
        for ctx, U, T in zip(self.ctxs, self.Us, self.Ts):
            nv.init_state(ctx, self.prim, U, T)
        t = torch.zeros(self.members, dtype=torch.float64, device=self.dev)
        e = nv.ensemble_create(self.ctxs, self.Us, self.Ts, lasers, t)
        half = self.nsteps // 2
        nv.run_ensemble(e, half, self.mode, dt_fixed=self.dt)
        mid = [nv.diagnostics(c, U, T)["heat_release"] for c, U, T in zip(self.ctxs, self.Us, self.Ts)]
        nv.run_ensemble(e, self.nsteps - half, self.mode, dt_fixed=self.dt)
        end = [nv.diagnostics(c, U, T) for c, U, T in zip(self.ctxs, self.Us, self.Ts)]
        del e
        return [d["max_T"] for d in end], mid, [d["heat_release"] for d in end]


def minimum_ignition_energy(runner: EnsembleIgnition, E_lo: float, E_hi: float, rounds: int = 4,
                            rtol: float = 0.0) -> Result:
    """Brackets the minimum ignition energy in [E_lo, E_hi] in at most `rounds`
    rounds (stopping once hi - lo <= rtol hi)."""
    lo, hi = float(E_lo), float(E_hi)
    res = Result((lo, hi))
    for _ in range(rounds):
        Es = probe_energies(lo, hi, runner.members)
        mT, hm, he = runner.run(Es)
        ok = [ignited(a, b, c, runner.T_fail) for a, b, c in zip(mT, hm, he)]
        lo, hi = next_bracket(Es, ok, lo, hi)
        res.rounds.append(Round(Es, ok, mT, hm, he, (lo, hi)))
        res.member_steps += runner.members * runner.nsteps
        if hi - lo <= rtol * hi:
            break
    res.bracket = (lo, hi)
    return res
