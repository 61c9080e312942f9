"""Shared helpers of the GPU parity tests: run the CUDA path and the oracle on
the same seeded inputs and compare."""
import gc

import numpy as np
import torch

import oracle
from oracle.mech import from_synth, grid_from_synth

F64 = torch.float64


def prim_tensor(case):
    return torch.as_tensor(case.prim, dtype=F64).cpu().contiguous()


def gpu_setup(case, precision=0, flags=0, options=None):
    from paper_2202_02319_b300 import native as nv
    gc.collect()            # release the constant-memory slots of mechanisms no longer referenced
    mech = nv.init_mechanism(case.mech)
    nodes = getattr(case, "nodes", None)
    if nodes is not None:
        flags |= nv.RF_MAPPED
    ctx = nv.create_ctx(mech, case.grid, precision, flags)
    if nodes is not None:
        nv.set_nodes(ctx, torch.as_tensor(np.ascontiguousarray(nodes), dtype=F64).cuda())
    for k, v in (options or {}).items():
        nv.set_option(ctx, k, v)
    ns = case.mech.n_species
    n = case.grid.ncells
    prim = prim_tensor(case).reshape(5 + ns, n).cuda()
    U = torch.empty((ns + 4, n), dtype=F64, device="cuda")
    T = torch.empty(n, dtype=F64, device="cuda")
    nv.init_state(ctx, prim, U, T)
    nv.check(ctx)
    nscbc_gpu(ctx, case)
    return mech, ctx, U, T


def nscbc_gpu(ctx, case):
    """Sets the case's characteristic-boundary sides on a context."""
    from paper_2202_02319_b300 import native as nv
    for (axis, side), spec in getattr(case, "nscbc", {}).items():
        kw = {k: v for k, v in spec.items() if k != "target"}
        tg = spec.get("target")
        if tg is not None:
            tg = torch.as_tensor(np.ascontiguousarray(tg), dtype=F64).cuda().contiguous()
        nv.set_nscbc(ctx, axis, side, target=tg, **kw)


def nscbc_oracle(case):
    """The oracle's 'nscbc' flags entry ({axis: {side: Side}}) of the case's sides."""
    g = case.grid
    out = {}
    for (axis, side), spec in getattr(case, "nscbc", {}).items():
        kw = {k: v for k, v in spec.items() if k != "target"}
        tg = spec.get("target")
        if tg is not None:
            plane = tuple(n for a, n in ((2, g.nz), (1, g.ny), (0, g.nx)) if a != axis)
            tg = torch.as_tensor(np.asarray(tg), dtype=F64).reshape((tg.shape[0],) + plane)
        out.setdefault(axis, {})[side] = oracle.nscbc.Side(target=tg, **kw)
    return out


def oracle_setup(case):
    mt = from_synth(case.mech)
    g = grid_from_synth(case.grid)
    nodes = getattr(case, "nodes", None)
    if nodes is not None:
        g = oracle.mapped.MappedGridT(g.nx, g.ny, g.nz, torch.as_tensor(np.asarray(nodes), dtype=F64), g.bc)
    U, T = oracle.rhs.init_state(mt, prim_tensor(case))
    return mt, g, U, T


def oracle_flags(flags):
    from paper_2202_02319_b300 import native as nv
    return {"inviscid": not (flags & nv.RF_NO_INVISCID), "viscous": not (flags & nv.RF_NO_VISCOUS),
            "chemistry": not (flags & nv.RF_NO_CHEMISTRY), "laser": not (flags & nv.RF_NO_LASER)}


def rel_inf(a, b):
    """Per-variable ||a_v - b_v||_inf / ||b_v||_inf (0/0 -> 0), as a numpy vector."""
    a = a.reshape(a.shape[0], -1).double().cpu()
    b = b.reshape(b.shape[0], -1).double().cpu()
    num = (a - b).abs().amax(1)
    den = b.abs().amax(1)
    return torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), num).numpy()


def rel_inf_group(a, b, ns):
    """Per-variable ||a_v - b_v||_inf over the largest |b| of the variable's group
    (species, momentum, energy), as a numpy vector: a variable whose values are all
    tiny (a species nothing produces yet) is measured against its group's scale
    (0/0 -> 0)."""
    a = a.reshape(a.shape[0], -1).double().cpu()
    b = b.reshape(b.shape[0], -1).double().cpu()
    num = (a - b).abs().amax(1)
    m = b.abs().amax(1)
    scale = torch.cat([m[:ns].max().repeat(ns), m[ns:ns + 3].max().repeat(3), m[ns + 3:]])
    return torch.where(scale > 0, num / torch.where(scale > 0, scale, torch.ones_like(scale)), num).numpy()


def rel_l2(a, b):
    a = a.reshape(a.shape[0], -1).double().cpu()
    b = b.reshape(b.shape[0], -1).double().cpu()
    num = (a - b).norm(dim=1)
    den = b.norm(dim=1)
    return torch.where(den > 0, num / torch.where(den > 0, den, torch.ones_like(den)), num).numpy()


def laser_tuple(case):
    return case.laser.as_tuple() if case.laser.E > 0 else None


def state_rel_l2(a, b, ns):
    """Relative L2 error of a conserved state, per variable, each scaled by the norm
    of its group: species densities by ||rho||, momentum components by ||rho |u|||,
    energy by ||E||.  (A per-species norm would divide by the near-zero densities
    of species a run has not produced yet.)"""
    a = a.reshape(a.shape[0], -1).double().cpu()
    b = b.reshape(b.shape[0], -1).double().cpu()
    rho = b[:ns].sum(0).norm()
    mom = b[ns:ns + 3].norm(dim=0).norm()
    scale = torch.cat([rho.repeat(ns), mom.repeat(3), b[ns + 3].norm().reshape(1)])
    return ((a - b).norm(dim=1) / scale).numpy()
