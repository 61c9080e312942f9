"""Throughput of the reacting-flow RHS / SSP-RK3 step on the 3-D jet-in-a-box
workload (256^3 cells, 9 species, 19 reversible reactions, Gaussian laser).

Metric: RHS cell-updates per second = cells x RHS evaluations / time (an RK3
step is three RHS evaluations plus the stage updates).  The headline `value` is
the mixed-precision path; the FP64 path is measured beside it (`fp64`).

One JSON line on rank 0.  Multi-GPU runs are independent replicas (the path
does not shard): each rank advances its own copy, value = all ranks' cell
updates / max-over-ranks time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--n 256] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "RHS cell-updates/s at 256^3 9 species, mixed vs FP64; % HBM roofline"
UNIT = "cell-updates/s"


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "source": "measured"}
    return {"hbm_gbs": 6400.0, "source": "fallback"}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# ----------------------------------------------------------------------------- algorithmic bytes

def sweep_bytes(ns: int, rsize: int, mode: str) -> int:
    """Algorithmic HBM bytes per cell of one sweep launch (each input read once,
    each output written once): Q fields (8 + 3 Ns), the state copy the fluxes use
    (FP32 copy in the mixed path, FP64 U otherwise), the RHS accumulator; the
    final sweep also reads U^n and U^(k) and writes U^(k+1) in FP64."""
    nv = ns + 4
    nq = 8 + 3 * ns
    b = nq * rsize + nv * rsize
    if mode == "accum":
        return b + 2 * nv * rsize
    return b + nv * rsize + 3 * nv * 8


def sweep_bytes_method(ns: int) -> int:
    """The fewest HBM bytes per cell a split flux sweep can move in FP32: the
    primitives u, v, w, T, p, c and Y_s (6 + Ns; rho follows from the equation of
    state), the coefficients mu, lambda and rho D_s (2 + Ns), and the RHS
    accumulator (4 + Ns) read and written: 208 B for 9 species."""
    return 4 * ((6 + ns) + (2 + ns)) + 2 * 4 * (ns + 4)


# Counts of the mixed-precision cell-state kernel (9 species, 19 reactions) from one
# ncu capture of the 96^3 jet case, per cell and averaged over the three launches of an
# RK step (the first also forms the chemical time-step rates: 209.0 DFMA, 69.0 DMUL,
# 15.0 DADD and 322.1 DRAM bytes; the other two 209.4, 69.1, 15.2 and 326.6): FP64
# thread instructions (DFMA, DMUL, DADD; FLOP = 2 DFMA + DMUL + DADD) and DRAM =
# dram__bytes_read.sum + dram__bytes_write.sum (traffic grows with the cell count, so a
# full 256^3 launch is the per-cell figure times 256^3).  Retaken with every change of
# the kernel.
CELL_STATE_MIXED_FP64_INST = (209.27, 69.08, 15.11)      # DFMA, DMUL, DADD per cell
CELL_STATE_MIXED_FP64_FLOP_PER_CELL = 2 * CELL_STATE_MIXED_FP64_INST[0] + sum(CELL_STATE_MIXED_FP64_INST[1:])
CELL_STATE_MIXED_DRAM_BYTES_PER_CELL = 325.1              # (322.1 + 2 x 326.6) / 3


def cell_state_bytes(ns: int, rsize: int) -> int:
    """Reads U (FP64) and T, writes T, the Q fields, the RHS source and (mixed) the FP32 copy of U."""
    nv = ns + 4
    b = nv * 8 + 8 + 8 + (8 + 3 * ns) * rsize + nv * rsize
    if rsize == 4:
        b += nv * 4
    return b


# ----------------------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    from paper_2202_02319_b300 import native as nv, synth
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n = args.n
    t_gen = time.time()
    case = synth.case_jet(0, n, device=dev)
    gen_s = time.time() - t_gen
    ns = case.mech.n_species
    ncell = case.grid.ncells
    prim = case.prim.reshape(5 + ns, ncell).contiguous()
    mech = nv.init_mechanism(case.mech)
    las = case.laser.as_tuple()

    def make(precision):
        ctx = nv.create_ctx(mech, case.grid, precision, 0)
        U = torch.empty((ns + 4, ncell), dtype=torch.float64, device=dev)
        T = torch.empty(ncell, dtype=torch.float64, device=dev)
        nv.init_state(ctx, prim, U, T)
        nv.check(ctx)
        return ctx, U, T

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed_steps(ctx, U, T, steps, warmup):
        t = torch.zeros(1, dtype=torch.float64, device=dev)
        dt = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(warmup):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, dt)
        nv.check(ctx)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(steps):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, dt)
        e1.record(s)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        nv.check(ctx)
        return ms, float(t), float(dt)

    # --- mixed path (headline)
    ctx, U, T = make(nv.RF_MIXED)
    with ClockSampler(local) as clk:
        ms_mixed, t_end, dt_last = timed_steps(ctx, U, T, args.steps, args.warmup)
    clocks = clk.summary()
    if world > 1:
        import torch.distributed as dist
        tm = torch.tensor([ms_mixed], device=dev)
        dist.all_reduce(tm, op=dist.ReduceOp.MAX)
        ms_mixed = float(tm)
    per_step_ms = ms_mixed / args.steps
    value = world * ncell * 3 * args.steps / (ms_mixed * 1e-3)
    launches_per_step = 0

    # per-kernel live timings (CUDA events on the launching stream) for one step
    nv.set_option(ctx, "profile", 1)
    tprof = torch.zeros(1, dtype=torch.float64, device=dev)
    tprof.fill_(t_end)
    nsteps_prof = 2
    for _ in range(nsteps_prof):
        nv.rk_step(ctx, U, T, tprof, 0.0, case.cfl, las, None)
    prof = nv.profile_read(ctx)
    nv.set_option(ctx, "profile", 0)
    launches_per_step = sum(v[1] for v in prof.values()) // nsteps_prof + 3     # + dt, prologue, epilogue kernels

    # --- e2e through the public host-buffer call: each step copies U, T in from pinned
    # host memory (by chunks overlapping the first stage) and U, T back out
    Uh = torch.empty_like(U, device="cpu").pin_memory()
    Th = torch.empty_like(T, device="cpu").pin_memory()
    Uh.copy_(U)
    Th.copy_(T)
    s = torch.cuda.current_stream()
    te = torch.zeros(1, dtype=torch.float64, device=dev)
    e2e_steps = max(1, min(args.e2e_steps, args.steps))
    nv.rk_step_host(ctx, Uh, Th, Uh, Th, te, 0.0, case.cfl, las, None)      # allocates the context's copies
    torch.cuda.synchronize()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(s)
    for _ in range(e2e_steps):
        nv.rk_step_host(ctx, Uh, Th, Uh, Th, te, 0.0, case.cfl, las, None)
    f1.record(s)
    torch.cuda.synchronize()
    nv.check(ctx)
    e2e_ms = f0.elapsed_time(f1)
    e2e_value = world * ncell * 3 * e2e_steps / (e2e_ms * 1e-3)
    h2d = (U.numel() + T.numel()) * 8
    d2h = (U.numel() + T.numel()) * 8
    del ctx, U, T, Uh, Th
    torch.cuda.empty_cache()

    # --- FP64 path
    ctx64, U64, T64 = make(nv.RF_FP64)
    ms64, _, _ = timed_steps(ctx64, U64, T64, args.fp64_steps, 1)
    nv.set_option(ctx64, "profile", 1)
    t64 = torch.zeros(1, dtype=torch.float64, device=dev)
    nv.rk_step(ctx64, U64, T64, t64, 0.0, case.cfl, las, None)
    prof64 = nv.profile_read(ctx64)
    nv.set_option(ctx64, "profile", 0)
    value64 = world * ncell * 3 * args.fp64_steps / (ms64 * 1e-3)
    del ctx64, U64, T64

    # --- TENO6 (the paper's sixth-order scheme) on the same workload, both precisions
    teno = run_teno_leg(args, mech, case, prim, dev) if args.teno_steps > 0 else None

    # --- characteristic-wise splitting with WENO3-Z and with TENO6, same workload
    charw = run_charwise_leg(args, mech, case, prim, dev) if args.charwise_steps > 0 else None

    # --- characteristic inflow / outflow boundaries: injection case, mixed
    nscbc = run_nscbc_leg(args, dev) if args.nscbc_steps > 0 else None

    # --- curvilinear grid: the jet on a curved periodic grid, mixed and FP64
    mapd = run_mapped_leg(args, dev) if args.mapped_steps > 0 else None

    # --- batched ensemble (64 members of uneven size): members/s per launch mode
    ens = run_ensemble_leg(args, dev) if args.ensemble_members > 0 else None

    # --- minimum ignition energy: bisection rounds over batched ensembles
    mie = run_mie_leg(args, dev) if args.mie_members > 0 else None

    # --- discrete adjoint: checkpointed ignition gradient of one 64^3 member (FP64)
    adj = run_adjoint_leg(args, dev) if args.adjoint_steps > 0 else None

    # --- roofline of the dominant kernel of the mixed step
    peaks = _peaks()
    fp64_peak = nv.probe_peak(0)
    fp32_peak = nv.probe_peak(1)
    tot = {k: v[0] for k, v in prof.items()}
    dom = max(("cell_state", "sweep_x", "sweep_y", "sweep_z"), key=lambda k: tot[k])
    kernels = {}
    prof["stage_update"] = prof["other"]
    tot["stage_update"] = tot["other"]
    for k in ("cell_state", "sweep_x", "sweep_y", "sweep_z", "stage_update"):
        ms_k, nl = prof[k]
        if nl == 0:
            continue
        avg = ms_k / nl
        if k == "cell_state":
            b = cell_state_bytes(ns, 4)
        elif k == "stage_update":
            # RHS (FP32) and U^(k) read, U^(k+1) written; U^n read in stages 2 and 3
            nv = ns + 4
            b = round(((nv * 4 + 2 * nv * 8) + 2 * (nv * 4 + 3 * nv * 8)) / 3, 1)
        else:
            # the mixed path's sweeps all accumulate; an elementwise kernel applies the stage
            b = sweep_bytes(ns, 4, "accum")
        gbs = b * ncell / (avg * 1e-3) / 1e9
        kernels[k] = {"ms_per_launch": round(avg, 4), "launches": nl,
                      "share": round(ms_k / sum(v for kk, v in tot.items() if kk != "stage_update"), 4),
                      "alg_bytes_per_cell": b, "achieved_gbs": round(gbs, 1),
                      "hbm_frac": round(gbs / peaks["hbm_gbs"], 4)}
        if k.startswith("sweep"):
            # the method's own minimum for a split sweep: 26 FP32 primitive and
            # coefficient fields read, the 13-variable FP32 RHS read and written
            bm = sweep_bytes_method(ns)
            gm = bm * ncell / (avg * 1e-3) / 1e9
            kernels[k].update({"method_bytes_per_cell": bm, "method_gbs": round(gm, 1),
                               "method_hbm_frac": round(gm / peaks["hbm_gbs"], 4)})
    k64 = {}
    for k in ("cell_state", "sweep_x", "sweep_y", "sweep_z"):
        ms_k, nl = prof64[k]
        if nl:
            k64[k] = {"ms_per_launch": round(ms_k / nl, 4), "share": round(ms_k / sum(v[0] for v in prof64.values()), 4)}
    d = kernels[dom]
    if dom == "cell_state" and CELL_STATE_MIXED_FP64_FLOP_PER_CELL:
        ms_k = prof["cell_state"][0] / prof["cell_state"][1]
        ach = CELL_STATE_MIXED_FP64_FLOP_PER_CELL * ncell / (ms_k * 1e-3) / 1e12
        traffic = (CELL_STATE_MIXED_DRAM_BYTES_PER_CELL * ncell) if CELL_STATE_MIXED_DRAM_BYTES_PER_CELL else None
        # the FP64 pipe issues one DFMA, DMUL or DADD per slot: instruction-issue fraction
        inst = sum(CELL_STATE_MIXED_FP64_INST)
        ach_i = inst * ncell / (ms_k * 1e-3) / 1e12
        roofline = {"kernel": dom, "bound": "alu", "achieved": round(ach, 4), "peak": round(fp64_peak, 4),
                    "unit": "TFLOP/s", "frac": round(ach / fp64_peak, 4), "traffic": traffic,
                    "peak_source": "FP64 FMA rate measured in this run (rf_probe_peak)",
                    "flop_per_cell": round(CELL_STATE_MIXED_FP64_FLOP_PER_CELL, 1),
                    "fp64_issue": {"inst_per_cell": round(inst, 1), "achieved_tinst_s": round(ach_i, 4),
                                   "peak_tinst_s": round(fp64_peak / 2, 4), "frac": round(ach_i / (fp64_peak / 2), 4)}}
    else:
        roofline = {"kernel": dom, "bound": "hbm", "achieved": d["achieved_gbs"], "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": d["hbm_frac"], "traffic": None,
                    "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs)"}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic (seeded jet-in-a-box, device-generated)",
        "config": {"workload": f"jet_in_box_{n}^3_9sp_19r_laser", "cells": ncell, "species": ns,
                   "reactions": case.mech.n_reactions, "precision": "mixed", "cfl": case.cfl,
                   "l2_flush": "not needed: state and workspace (>10 GB) exceed the 126 MB L2",
                   "parallelism": f"replicas x{world}"},
        "fp64": {"value": value64, "unit": UNIT, "ms_per_step": ms64 / args.fp64_steps, "steps": args.fp64_steps,
                 "kernels": k64},
        "kernels": kernels,
        "roofline": roofline,
        "teno6": teno,
        "charwise": charw,
        "nscbc": nscbc,
        "mapped": mapd,
        "min_ignition_energy": mie,
        "ensemble": ens,
        "adjoint": adj,
        "peaks_measured": {"fp64_tflops": round(fp64_peak, 4), "fp32_tflops": round(fp32_peak, 3),
                           "hbm_gbs": peaks["hbm_gbs"], "hbm_source": peaks["source"]},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "sim": {"t_end_s": t_end, "dt_last_s": dt_last, "generation_s": round(gen_s, 2)},
    }
    if rank == 0 and not args.no_cpu_baseline:
        case.prim = prim.reshape(case.prim.shape)
        out["cpu_baseline"] = cpu_baseline(case, block=args.cpu_n, full=args.cpu_full)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ----------------------------------------------------------------------------- TENO6 leg

def run_teno_leg(args, mech, case, prim, dev, flags=None, steps_mixed=None):
    """Cell-updates/s of the same workload with the inviscid fluxes by TENO6 (six-cell
    stencils, sweeps from global memory), or with the scheme `flags` selects, mixed
    and FP64, CUDA events on the launching stream, per-kernel times from the
    library's profile events."""
    import torch
    from paper_2202_02319_b300 import native as nv
    ns = case.mech.n_species
    ncell = case.grid.ncells
    las = case.laser.as_tuple()
    flags = nv.RF_TENO6 if flags is None else flags
    steps_mixed = args.teno_steps if steps_mixed is None else steps_mixed
    out = {}
    for name, prec, steps in (("mixed", nv.RF_MIXED, steps_mixed), ("fp64", nv.RF_FP64, max(1, steps_mixed // 2))):
        ctx = nv.create_ctx(mech, case.grid, prec, flags)
        U = torch.empty((ns + 4, ncell), dtype=torch.float64, device=dev)
        T = torch.empty(ncell, dtype=torch.float64, device=dev)
        nv.init_state(ctx, prim, U, T)
        t = torch.zeros(1, dtype=torch.float64, device=dev)
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        nv.check(ctx)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(steps):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nv.set_option(ctx, "profile", 1)
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        prof = nv.profile_read(ctx)
        nv.set_option(ctx, "profile", 0)
        nv.check(ctx)
        out[name] = {"value": ncell * 3 * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps,
                     "steps": steps,
                     "kernels_ms_per_launch": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]}}
        del ctx, U, T
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- characteristic-wise leg

def run_charwise_leg(args, mech, case, prim, dev):
    """The same workload with characteristic-wise splitting (RF_CHARWISE), WENO3-Z and
    TENO6, mixed and FP64."""
    from paper_2202_02319_b300 import native as nv
    return {"weno3z": run_teno_leg(args, mech, case, prim, dev, nv.RF_CHARWISE, args.charwise_steps),
            "teno6": run_teno_leg(args, mech, case, prim, dev, nv.RF_CHARWISE | nv.RF_TENO6, args.charwise_steps)}


# ----------------------------------------------------------------------------- NSCBC leg

def run_nscbc_leg(args, dev):
    """Injection through characteristic boundaries (x inflow / outflow, y and z
    zero-gradient) on an nx x ny x ny box, mixed precision: cell-updates/s, and the
    same grid with zero-gradient x ends, so the difference is the boundary kernels'
    cost (their time per step from the profile's 'other' class, less the stage
    updates')."""
    import torch
    from paper_2202_02319_b300 import native as nv, synth
    nx, ny = args.nscbc_nx, args.nscbc_ny
    case = synth.case_jet_inflow(0, nx, ny, ny)
    ns = case.mech.n_species
    ncell = case.grid.ncells
    mech = nv.init_mechanism(case.mech)
    prim = torch.as_tensor(case.prim, dtype=torch.float64).reshape(5 + ns, ncell).to(dev)
    out = {"grid": [nx, ny, ny], "cells": ncell, "steps": args.nscbc_steps}
    for name, bcx in (("nscbc", synth.BC_NSCBC), ("zero_gradient", synth.BC_EXTRAPOLATE)):
        grid = synth.Grid(nx, ny, ny, case.grid.dx, case.grid.dy, case.grid.dz, (bcx,) + tuple(case.grid.bc[1:]))
        ctx = nv.create_ctx(mech, grid, nv.RF_MIXED)
        if bcx == synth.BC_NSCBC:
            for (axis, side), spec in case.nscbc.items():
                kw = {k: v for k, v in spec.items() if k != "target"}
                tg = spec.get("target")
                tg = torch.as_tensor(tg, dtype=torch.float64).to(dev).contiguous() if tg is not None else None
                nv.set_nscbc(ctx, axis, side, target=tg, **kw)
        U = torch.empty((ns + 4, ncell), dtype=torch.float64, device=dev)
        T = torch.empty(ncell, dtype=torch.float64, device=dev)
        nv.init_state(ctx, prim, U, T)
        t = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(2):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, None, None)
        nv.check(ctx)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(args.nscbc_steps):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, None, None)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nv.set_option(ctx, "profile", 1)
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, None, None)
        prof = nv.profile_read(ctx)
        nv.set_option(ctx, "profile", 0)
        nv.check(ctx)
        out[name] = {"value": ncell * 3 * args.nscbc_steps / (ms * 1e-3), "unit": UNIT,
                     "ms_per_step": ms / args.nscbc_steps, "other_ms_per_step": prof["other"][0],
                     "other_launches_per_step": prof["other"][1]}
        del ctx, U, T
        torch.cuda.empty_cache()
    out["boundary_kernels_ms_per_step"] = round(out["nscbc"]["other_ms_per_step"] - out["zero_gradient"]["other_ms_per_step"], 4)
    out["step_time_ratio"] = round(out["nscbc"]["ms_per_step"] / out["zero_gradient"]["ms_per_step"], 4)
    return out


# ----------------------------------------------------------------------------- mapped-grid leg

def run_mapped_leg(args, dev):
    """The jet in a box on a curved periodic grid (synth.case_jet_mapped, n^3), mixed
    and FP64: cell-updates/s with CUDA events on the launching stream, per-kernel
    times from the library's profile events."""
    import torch
    from paper_2202_02319_b300 import native as nv, synth
    case = synth.case_jet_mapped(0, args.mapped_n)
    ns = case.mech.n_species
    ncell = case.grid.ncells
    mech = nv.init_mechanism(case.mech)
    prim = torch.as_tensor(case.prim, dtype=torch.float64).reshape(5 + ns, ncell).to(dev)
    nodes = torch.as_tensor(case.nodes, dtype=torch.float64).to(dev).contiguous()
    las = case.laser.as_tuple()
    out = {"grid": [args.mapped_n] * 3, "cells": ncell, "amplitude_cells": 0.2}
    for name, prec, steps in (("mixed", nv.RF_MIXED, args.mapped_steps), ("fp64", nv.RF_FP64, max(1, args.mapped_steps // 2))):
        ctx = nv.create_ctx(mech, case.grid, prec, nv.RF_MAPPED)
        nv.set_nodes(ctx, nodes)
        U = torch.empty((ns + 4, ncell), dtype=torch.float64, device=dev)
        T = torch.empty(ncell, dtype=torch.float64, device=dev)
        nv.init_state(ctx, prim, U, T)
        t = torch.zeros(1, dtype=torch.float64, device=dev)
        for _ in range(2):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        nv.check(ctx)
        s = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        for _ in range(steps):
            nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        nv.set_option(ctx, "profile", 1)
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, None)
        prof = nv.profile_read(ctx)
        nv.set_option(ctx, "profile", 0)
        nv.check(ctx)
        out[name] = {"value": ncell * 3 * steps / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms / steps, "steps": steps,
                     "kernels_ms_per_launch": {k: round(v[0] / v[1], 4) for k, v in prof.items() if v[1]}}
        del ctx, U, T
        torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- ignition leg

def run_mie_leg(args, dev):
    """Minimum-ignition-energy bisection: `mie_members` copies of the jet state at
    `mie_n`^3 per round, laser energies spread in the bracket, one batched
    ensemble (CUDA graph, mixed precision) per round; members/s of the search."""
    import time
    import torch
    from paper_2202_02319_b300 import ignition, native as nv, synth
    case = synth.case_jet(0, args.mie_n)
    case.laser.t0 = 2e-8
    runner = ignition.EnsembleIgnition(case, args.mie_members, args.mie_steps, 1e-9, precision=nv.RF_MIXED,
                                       mode=nv.ENS_GRAPH, device=dev)
    runner.run([case.laser.E] * args.mie_members)          # warm-up (captures the graphs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res = ignition.minimum_ignition_energy(runner, 1e-3, 40e-3, rounds=args.mie_rounds)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    n = len(res.rounds) * args.mie_members
    return {"members": args.mie_members, "cells_per_member": case.grid.ncells, "steps": args.mie_steps,
            "rounds": len(res.rounds), "bracket_J": list(res.bracket), "seconds": round(el, 3),
            "members_per_s": n / el, "cell_updates_per_s": n * case.grid.ncells * 3 * args.mie_steps / el,
            "timing": "host clock around synchronised rounds (ensemble set-up and diagnostics included)"}


# ----------------------------------------------------------------------------- adjoint leg

def run_adjoint_leg(args, dev):
    """Gradient of the time-integrated heat release with respect to (E, x0, y0, z0,
    sigma_r, ln A_j) for jet members of n^3 cells, each with its own laser: forward
    run with a checkpoint every `adjoint_ck` steps, then the reverse sweep
    (recomputation within segments, RK-step adjoints), both FP64.  The pulse is
    centred inside the window so that every laser gradient is nonzero."""
    import time
    import torch
    from paper_2202_02319_b300 import adjoint, synth
    n, nsteps, dt, nm = args.adjoint_n, args.adjoint_steps, 1e-9, max(1, args.adjoint_members)
    cases = synth.adjoint_members(0, nm, n, t0=0.5 * nsteps * dt)
    ck = args.adjoint_ck if args.adjoint_ck > 0 else max(1, nsteps // 2)
    probs = [adjoint.HeatReleaseProblem(c.mech, c.grid, c.prim, c.laser, nsteps=nsteps, dt=dt,
                                        checkpoint_every=ck, device=dev, store_stages=not args.adjoint_recompute)
             for c in cases]
    p0 = [pr.default_params() for pr in probs]
    probs[0].run(p0[0], keep=False)               # warm-up (also builds the kernels' first launches)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for pr, p in zip(probs, p0):
        pr.run(p, keep=False)
    torch.cuda.synchronize()
    t_fwd = time.perf_counter() - t0
    t0 = time.perf_counter()
    grads, Js = [], []
    for pr, p in zip(probs, p0):
        J, st = pr.run_with_state(p)
        grads.append(pr.gradient(st))
        Js.append(J)
    torch.cuda.synchronize()
    t_grad = time.perf_counter() - t0
    cells = cases[0].grid.ncells
    return {"members": nm, "cells": cells, "steps": nsteps, "dt_s": dt, "checkpoint_every": ck,
            "stages": "recomputed" if args.adjoint_recompute else "stored within each segment",
            "params": int(p0[0].numel()),
            "forward_ms": round(t_fwd * 1e3, 2), "forward_and_gradient_ms": round(t_grad * 1e3, 2),
            "gradient_over_forward": round(t_grad / t_fwd, 2),
            "members_per_s_gradient": nm / t_grad,
            "cell_updates_per_s_forward": nm * cells * 3 * nsteps / t_fwd, "J": Js[0],
            "dJ_dE": float(grads[0][0]), "timing": "host clock around synchronised calls, FP64"}


# ----------------------------------------------------------------------------- ensemble leg

def run_ensemble_leg(args, dev):
    """Members/s of the batched-ensemble workload (members with every axis in
    U{48..96}, laser energy U[5, 40] mJ) in the mixed path: the per-member launch
    loop against one launch per phase in a CUDA graph and one persistent launch
    per RK stage in a CUDA graph, after autotuning the walk segment."""
    import torch
    from paper_2202_02319_b300 import native as nv, synth
    cases = synth.ensemble_members(seed=0, n_members=args.ensemble_members, device=dev)
    mech = nv.init_mechanism(cases[0].mech)
    ctxs, Us, Ts = [], [], []
    for c in cases:
        ns, n = c.mech.n_species, c.grid.ncells
        ctx = nv.create_ctx(mech, c.grid, nv.RF_MIXED)
        U = torch.empty((ns + 4, n), dtype=torch.float64, device=dev)
        T = torch.empty(n, dtype=torch.float64, device=dev)
        nv.init_state(ctx, c.prim.reshape(5 + ns, n).contiguous(), U, T)
        ctxs.append(ctx)
        Us.append(U)
        Ts.append(T)
        c.prim = None
    t = torch.zeros(len(cases), dtype=torch.float64, device=dev)
    e = nv.ensemble_create(ctxs, Us, Ts, [c.laser.as_tuple() for c in cases], t)
    seg = nv.ensemble_autotune(e, nv.ENS_GRAPH, 0.5)
    cells = sum(c.grid.ncells for c in cases)
    out = {"members": len(cases), "cells": cells, "walk_seg_autotuned": seg, "steps": args.ensemble_steps}
    s = torch.cuda.current_stream()
    for name, mode in (("member_loop", nv.ENS_LOOP), ("batched_graph", nv.ENS_GRAPH),
                       ("persistent", nv.ENS_PERSISTENT)):
        nv.run_ensemble(e, 1, mode, 0.5)                 # warm-up (captures the graph)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s)
        code, st = nv.run_ensemble(e, args.ensemble_steps, mode, 0.5, raise_on_error=False)
        e1.record(s)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"members_per_s": len(cases) * args.ensemble_steps / (ms * 1e-3),
                     "cell_updates_per_s": cells * 3 * args.ensemble_steps / (ms * 1e-3),
                     "ms_per_step": ms / args.ensemble_steps, "failed_members": sum(1 for x in st if x)}
    out["speedup_persistent_vs_loop"] = out["persistent"]["members_per_s"] / out["member_loop"]["members_per_s"]
    out["speedup_batched_vs_loop"] = out["batched_graph"]["members_per_s"] / out["member_loop"]["members_per_s"]
    del e, ctxs, Us, Ts
    torch.cuda.empty_cache()
    return out


# ----------------------------------------------------------------------------- oracle arm

def workload_block(prim, grid, b):
    """A b^3 block of the workload's primitive fields (on the host), centred on the
    jet axis (y, z) and the middle of the box in x, with zero-gradient ghost
    cells: the same state, mechanism and per-cell work as the full box."""
    import torch
    nz, ny, nx = prim.shape[1:]
    b = min(b, nx, ny, nz)
    z0, y0, x0 = (nz - b) // 2, (ny - b) // 2, (nx - b) // 2
    blk = prim[:, z0:z0 + b, y0:y0 + b, x0:x0 + b].to("cpu", torch.float64).contiguous()
    from oracle.mech import GridT
    return blk, GridT(b, b, b, grid.dx, grid.dy, grid.dz, (1, 1, 1))


def _time_oracle_rhs(mt, g, prim, las, budget_s, min_evals=2, max_evals=1000):
    import oracle
    U, T = oracle.rhs.init_state(mt, prim)
    oracle.rhs.rhs(mt, g, U, T, 0.0, las)            # warm-up
    t0 = time.time()
    k = 0
    while k < max_evals and (k < min_evals or time.time() - t0 < budget_s):
        oracle.rhs.rhs(mt, g, U, T, 0.0, las)
        k += 1
    return k, time.time() - t0


def cpu_baseline(case, block=64, block1=24, budget_s=12.0, budget1_s=6.0, full=False):
    """The oracle as it stands (vectorised torch-CPU FP64) timed on the host cores,
    on blocks of the workload itself: all threads on a `block`^3 block, one thread
    on a `block1`^3 block; with `full`, one RHS on the whole box as well."""
    import torch
    from oracle.mech import from_synth
    mt = from_synth(case.mech)
    las = case.laser.as_tuple()
    ns = case.mech.n_species
    prim = case.prim.reshape(5 + ns, case.grid.nz, case.grid.ny, case.grid.nx)
    cores = len(os.sched_getaffinity(0))
    threads = torch.get_num_threads()
    blk, g = workload_block(prim, case.grid, block)
    k, el = _time_oracle_rhs(mt, g, blk, las, budget_s)
    ncell = g.nx * g.ny * g.nz
    out = {"value": ncell * k / el, "unit": UNIT, "cores": threads, "host_cores": cores, "kind": "oracle",
           "sample": f"{k} oracle RHS evaluations on a {g.nx}^3 block of the {case.grid.nx}^3 workload "
                     f"(centred on the jet, zero-gradient edges) in {el:.1f} s on {threads} threads"}
    blk1, g1 = workload_block(prim, case.grid, block1)
    torch.set_num_threads(1)
    try:
        k1, el1 = _time_oracle_rhs(mt, g1, blk1, las, budget1_s)
    finally:
        torch.set_num_threads(threads)
    out["single_core"] = {"value": g1.nx * g1.ny * g1.nz * k1 / el1, "unit": UNIT, "threads": 1,
                          "sample": f"{k1} oracle RHS evaluations on a {g1.nx}^3 block in {el1:.1f} s"}
    if full:
        import oracle
        from oracle.mech import grid_from_synth
        gf = grid_from_synth(case.grid)
        Uf, Tf = oracle.rhs.init_state(mt, prim.to("cpu", torch.float64))
        t0 = time.time()
        oracle.rhs.rhs(mt, gf, Uf, Tf, 0.0, las)
        elf = time.time() - t0
        out["full_box"] = {"value": case.grid.ncells / elf, "unit": UNIT, "threads": threads,
                           "sample": f"one oracle RHS on the whole {case.grid.nx}^3 box in {elf:.1f} s"}
    return out


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    import torch
    from paper_2202_02319_b300 import synth
    from oracle.mech import from_synth
    case = synth.case_jet(0, args.n)                 # the same generator, on the host
    mt = from_synth(case.mech)
    las = case.laser.as_tuple()
    ns = case.mech.n_species
    prim = case.prim.reshape(5 + ns, case.grid.nz, case.grid.ny, case.grid.nx)
    blk, g = workload_block(prim, case.grid, args.cpu_n)
    import oracle
    U, T = oracle.rhs.init_state(mt, blk)
    for _ in range(args.warmup):
        oracle.rhs.rhs(mt, g, U, T, 0.0, las)
    t0 = time.time()
    for _ in range(args.steps):
        oracle.rhs.rhs(mt, g, U, T, 0.0, las)
    el = time.time() - t0
    ncell = g.nx * g.ny * g.nz
    value = ncell * args.steps / el
    threads = torch.get_num_threads()
    cb = {"value": value, "unit": UNIT, "cores": threads, "host_cores": len(os.sched_getaffinity(0)),
          "kind": "oracle",
          "sample": f"each step one oracle RHS evaluation on a {g.nx}^3 block of the {args.n}^3 workload "
                    f"(centred on the jet, zero-gradient edges); {args.steps} steps in {el:.1f} s"}
    out = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": el * 1e3 / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic (seeded jet-in-a-box, host-generated)",
           "config": {"workload": f"jet_in_box_{args.n}^3_9sp_19r_laser", "cells": case.grid.ncells,
                      "species": ns, "reactions": case.mech.n_reactions, "precision": "fp64 (oracle)",
                      "sample_block": f"{g.nx}^3"},
           "cpu_baseline": cb,
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--cpu-n", type=int, default=64)
    ap.add_argument("--cpu-full", action="store_true", help="also time one oracle RHS on the whole box")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--teno-steps", type=int, default=4)
    ap.add_argument("--charwise-steps", type=int, default=2)
    ap.add_argument("--mapped-steps", type=int, default=4)
    ap.add_argument("--mapped-n", type=int, default=192)
    ap.add_argument("--nscbc-steps", type=int, default=10)
    ap.add_argument("--nscbc-nx", type=int, default=256)
    ap.add_argument("--nscbc-ny", type=int, default=128)
    ap.add_argument("--mie-members", type=int, default=8)
    ap.add_argument("--mie-n", type=int, default=48)
    ap.add_argument("--mie-steps", type=int, default=40)
    ap.add_argument("--mie-rounds", type=int, default=2)
    ap.add_argument("--ensemble-members", type=int, default=64)
    ap.add_argument("--ensemble-steps", type=int, default=10)
    ap.add_argument("--adjoint-n", type=int, default=64)
    ap.add_argument("--adjoint-steps", type=int, default=20)
    ap.add_argument("--adjoint-members", type=int, default=1)
    ap.add_argument("--adjoint-ck", type=int, default=0, help="checkpoint interval (0: half the steps)")
    ap.add_argument("--adjoint-recompute", action="store_true",
                    help="recompute every step's stages in the reverse sweep instead of keeping them")
    ap.add_argument("--leg", default=None, choices=["mapped", "nscbc", "charwise"],
                    help="run only this leg and print its result (for profiling its kernels)")
    args = ap.parse_args()
    if args.leg is not None:
        import torch
        dev = torch.device("cuda")
        if args.leg == "charwise":
            from paper_2202_02319_b300 import native as nv, synth
            case = synth.case_jet(0, args.n, device=dev)
            prim = case.prim.reshape(5 + case.mech.n_species, case.grid.ncells).contiguous()
            leg = run_charwise_leg(args, nv.init_mechanism(case.mech), case, prim, dev)
        else:
            leg = run_mapped_leg(args, dev) if args.leg == "mapped" else run_nscbc_leg(args, dev)
        print(json.dumps({"leg": args.leg, **leg}))
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
