"""State error against the FP64 oracle at the sizes of the configured workloads,
reported as JSON (one line per leg).  The oracle legs run in a worker process
(started with `spawn` before any CUDA call) while the GPU legs run here.

Legs (paper: Methods - Diffusion flame and Model rocket combustor set up the two
workloads the mixing layer and the jet in a box stand in for):
  c1  32^3 box, 4 species / 3 reactions: 10 SSP-RK3 steps at the time-step rule
      (CFL 0.5), FP64 against the oracle (each side applies the rule itself) and
      mixed against the oracle (on the oracle's dt sequence).
  c2  512 x 512 mixing layer, 9 species / 19 reactions: 200 steps of dt = 5 ns,
      FP64 and mixed against the oracle.
  c3  jet in a box: the 256^3 workload, 100 steps of dt = 1 ns with the pulse
      inside the window, mixed against FP64 (both on the GPU; the FP64 path matches
      the oracle to 1e-12 per RHS); and the same generator at 64^3, FP64 and mixed
      against the oracle over the same 100 steps.
  c4  the two smallest of the 64 ensemble members (48^3 to 96^3), pulses inside
      the window: 100 steps of dt = 1 ns in one persistent launch per RK stage and
      in the batched graph, each member against the oracle.
Errors: per conserved variable ||U - U_oracle||_2, divided by its group's norm
(species by ||rho||, momentum by ||rho |u|||, energy by ||E||); `max` is the
largest over the variables.  Bars: FP64 1e-10, mixed and ensemble 1e-5.

  python tests/config_parity.py [--legs c1,c2,c3,c4]
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _leg_cases(leg):
    from paper_2202_02319_b300 import synth
    if leg == "c1":
        return {"box32": synth.case_box32(0)}
    if leg == "c2":
        return {"mixing512": synth.case_mixing_layer(0, 512)}
    if leg == "c3":
        c = synth.case_jet(0, 64)
        c.laser.t0 = 5e-8
        return {"jet64": c}
    if leg == "c4":
        cases = synth.ensemble_members(seed=0, n_members=64)
        cases = sorted(cases, key=lambda c: c.grid.ncells)[:2]
        for c in cases:
            c.laser.t0 = 5e-8
        return {c.name: c for c in cases}
    raise ValueError(leg)


LEG_STEPS = {"c1": (10, 0.0), "c2": (200, 5e-9), "c3": (100, 1e-9), "c4": (100, 1e-9)}


def _oracle_worker(legs, q):
    """Runs the oracle legs in order; puts (leg, name, U, dts, seconds) per case."""
    import torch
    import oracle
    from oracle.mech import from_synth, grid_from_synth
    torch.set_num_threads(max(1, len(os.sched_getaffinity(0))))
    for leg in legs:
        nsteps, dt = LEG_STEPS[leg]
        for name, case in _leg_cases(leg).items():
            t0 = time.time()
            mt, g = from_synth(case.mech), grid_from_synth(case.grid)
            U, T = oracle.rhs.init_state(mt, torch.as_tensor(case.prim, dtype=torch.float64))
            las = case.laser.as_tuple() if case.laser.E > 0 else None
            t, dts = 0.0, []
            for _ in range(nsteps):
                U, T, d = oracle.rk.rk_step(mt, g, U, T, t, dt, las, 0.5)
                dts.append(d)
                t += d
            q.put((leg, name, U.reshape(U.shape[0], -1).numpy(), dts, time.time() - t0))
    q.put(None)


def _err(a, b, ns):
    from tests.gpu_common import state_rel_l2
    e = state_rel_l2(a, b, ns)
    return {"max": float(e.max()), "per_variable": [float(x) for x in e]}


def _gpu_single(case, precision, nsteps, dt, dts=None):
    import torch
    from paper_2202_02319_b300 import native as nv
    from tests.gpu_common import gpu_setup
    mech, ctx, U, T = gpu_setup(case, precision=precision)
    las = case.laser.as_tuple() if case.laser.E > 0 else None
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for k in range(nsteps):
        d = dts[k] if dts is not None else dt
        nv.rk_step(ctx, U, T, t, d, 0.5, las, None)
    nv.check(ctx)
    return U


def _gpu_ensemble(cases, mode, nsteps, dt):
    import torch
    from paper_2202_02319_b300 import native as nv
    mech = nv.init_mechanism(cases[0].mech)
    ctxs, Us, Ts = [], [], []
    for c in cases:
        ns, n = c.mech.n_species, c.grid.ncells
        ctx = nv.create_ctx(mech, c.grid, nv.RF_MIXED)
        U = torch.empty((ns + 4, n), dtype=torch.float64, device="cuda")
        T = torch.empty(n, dtype=torch.float64, device="cuda")
        nv.init_state(ctx, torch.as_tensor(c.prim, dtype=torch.float64).reshape(5 + ns, n).cuda(), U, T)
        ctxs.append(ctx)
        Us.append(U)
        Ts.append(T)
    t = torch.zeros(len(cases), dtype=torch.float64, device="cuda")
    e = nv.ensemble_create(ctxs, Us, Ts, [c.laser.as_tuple() for c in cases], t)
    code, st = nv.run_ensemble(e, nsteps, mode, dt_fixed=dt)
    assert code == 0 and not any(st), (code, st)
    return Us


def _c3_fullsize():
    """Mixed against FP64 on the 256^3 workload, both on the GPU."""
    import torch
    from paper_2202_02319_b300 import native as nv, synth
    from tests.gpu_common import state_rel_l2
    case = synth.case_jet(0, 256, device="cuda")
    case.laser.t0 = 5e-8
    t0 = time.time()
    U64 = _gpu_single(case, nv.RF_FP64, 100, 1e-9).cpu()
    torch.cuda.empty_cache()
    Umx = _gpu_single(case, nv.RF_MIXED, 100, 1e-9).cpu()
    e = state_rel_l2(Umx, U64, case.mech.n_species)
    return {"leg": "c3", "case": "jet256_mixed_vs_fp64_gpu", "steps": 100, "dt_s": 1e-9,
            "mixed_vs_fp64": {"max": float(e.max()), "per_variable": [float(x) for x in e]},
            "bar": 1e-5, "seconds": round(time.time() - t0, 1)}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--legs", default="c1,c2,c3,c4")
    args = ap.parse_args()
    legs = [x for x in args.legs.split(",") if x]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    worker = ctx.Process(target=_oracle_worker, args=(legs, q))
    worker.start()                     # before any CUDA call in this process
    import torch
    from paper_2202_02319_b300 import native as nv
    if "c3" in legs:
        print(json.dumps(_c3_fullsize()), flush=True)
    while True:
        item = q.get()
        if item is None:
            break
        leg, name, Uo, dts, secs = item
        Uo = torch.as_tensor(Uo)
        nsteps, dt = LEG_STEPS[leg]
        case = _leg_cases(leg)[name]
        ns = case.mech.n_species
        out = {"leg": leg, "case": name, "cells": case.grid.ncells, "steps": nsteps,
               "dt_s": dt if dt > 0 else "rule (CFL 0.5)", "oracle_seconds": round(secs, 1)}
        if leg == "c4":
            cases = list(_leg_cases(leg).values())
            idx = [c.name for c in cases].index(name)
            for label, mode in (("persistent", nv.ENS_PERSISTENT), ("batched_graph", nv.ENS_GRAPH)):
                Us = _gpu_ensemble(cases, mode, nsteps, dt)
                out[label] = _err(Us[idx], Uo, ns)
            out["bar"] = 1e-5
        else:
            out["fp64"] = _err(_gpu_single(case, nv.RF_FP64, nsteps, dt), Uo, ns)
            out["mixed"] = _err(_gpu_single(case, nv.RF_MIXED, nsteps, dt, dts if dt <= 0 else None), Uo, ns)
            out["bars"] = {"fp64": 1e-10, "mixed": 1e-5}
        print(json.dumps(out), flush=True)
        torch.cuda.empty_cache()
    worker.join()
    return 0 if worker.exitcode == 0 else 1


if __name__ == "__main__":
    sys.exit(main())
