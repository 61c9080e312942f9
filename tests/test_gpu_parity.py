"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on the same
seeded inputs.  Bar: FP64 path within 1e-12 of the oracle per conserved
variable (max-norm relative to the variable's max magnitude); mixed path within
1e-5 relative L2 after a run of steps."""
import math

import numpy as np
import pytest
import torch

import oracle
from oracle.mech import GridT
from paper_2202_02319_b300 import synth
from tests.gpu_common import (gpu_setup, laser_tuple, oracle_flags, oracle_setup, prim_tensor, rel_inf, rel_l2,
                              state_rel_l2)
from tests.helpers import random_prim, single_species

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _random_case(shape, bc, seed, mk=synth.mechanism_9sp, smooth=False):
    m = mk(seed)
    nz, ny, nx = shape
    grid = synth.Grid(nx, ny, nz, 1.1e-4, 0.9e-4, 1.3e-4, bc)
    return synth.Case(f"random{shape}", m, grid, random_prim(m, shape, seed, smooth=smooth))


def _cases():
    c = [synth.case_box32(0), synth.case_jet(0, 16), synth.case_mixing_layer(0, 32),
         _random_case((5, 7, 13), (1, 0, 1), 3), _random_case((6, 5, 1), (0, 0, 0), 4),
         _random_case((1, 1, 1), (0, 0, 0), 5), _random_case((4, 9, 300), (0, 1, 0), 6, smooth=True),
         _random_case((3, 4, 256), (0, 0, 1), 7, smooth=True)]
    jet = c[1]
    jet.laser.t0 = 2e-8           # laser on at t = 0
    jet.laser.x0 = 8.3 * jet.grid.dx
    jet.laser.y0 = 7.6 * jet.grid.dx
    jet.laser.z0 = 8.1 * jet.grid.dx
    return c


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_init_state_parity(case):
    _, _, U, T = gpu_setup(case)
    _, _, Uo, To = oracle_setup(case)
    assert rel_inf(U, Uo.reshape(U.shape)).max() < 4e-15
    assert torch.equal(T.cpu(), To.reshape(-1))


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_rhs_parity_fp64(case):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case)
    out = torch.empty_like(U)
    las = laser_tuple(case)
    nv.rhs(ctx, U, T, 0.0, las, out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    ro, Tn = oracle.rhs.rhs(mt, g, Uo, To, 0.0, las)
    err = rel_inf(out, ro)
    assert err.max() < TOL64, err
    assert rel_inf(T[None], Tn.reshape(1, -1)).max() < 1e-14


@pytest.mark.parametrize("flags", [1, 2, 4, 8, 6])
def test_rhs_parity_term_switches(flags):
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=flags)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, laser_tuple(case), oracle_flags(flags))
    assert rel_inf(out, ro).max() < TOL64


@pytest.mark.parametrize("opts", [{"x_block": 64}, {"x_block": 32, "walk_seg": 1}, {"walk_seg": 5, "walk_block": 32}])
def test_launch_shapes_do_not_change_results(opts):
    """The x sweep's row chunking and the y/z walk segmentation are bitwise
    invisible: different launch shapes give identical RHS."""
    nv = _nv()
    case = _random_case((5, 13, 100), (0, 1, 0), 11, smooth=True)
    res = []
    for o in ({}, opts):
        mech, ctx, U, T = gpu_setup(case, options=o)
        out = torch.empty_like(U)
        nv.rhs(ctx, U, T, 0.0, None, out)
        nv.check(ctx)
        res.append(out.cpu())
    assert torch.equal(res[0], res[1])


def test_uniform_state_rhs_is_exactly_zero():
    nv = _nv()
    m = synth.mechanism_9sp(0)
    Y = np.random.default_rng(0).dirichlet(np.ones(9))
    vals = np.concatenate([[1.3e5, 900.0, 37.0, -12.0, 5.0], Y])
    case = synth.Case("uniform", m, synth.Grid(7, 6, 5, 1e-4, 2e-4, 1.5e-4), vals.reshape(-1, 1, 1, 1) * np.ones((1, 5, 6, 7)))
    for prec in (nv.RF_FP64, nv.RF_MIXED):
        mech, ctx, U, T = gpu_setup(case, precision=prec, flags=nv.RF_NO_CHEMISTRY)
        out = torch.empty_like(U)
        nv.rhs(ctx, U, T, 0.0, None, out)
        nv.check(ctx)
        assert float(out.abs().max()) == 0.0


@pytest.mark.parametrize("idx", [0, 1, 2, 5])
def test_rk_step_parity_fp64(idx):
    """Three SSP-RK3 steps with the time-step rule: dt and state match the oracle."""
    nv = _nv()
    case = CASES[idx]
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    las = laser_tuple(case)
    to = 0.0
    for _ in range(3):
        nv.rk_step(ctx, U, T, t, 0.0, case.cfl, las, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, las, case.cfl)
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
        assert abs(float(t) - to) <= 1e-12 * to
    assert rel_inf(U, Uo).max() < TOL64


def test_mixed_precision_l2_after_steps():
    """Mixed path vs the FP64 oracle: relative L2 per conserved variable (scaled by
    its group's norm) after 10 steps of the 32^3 box stays below 1e-5."""
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    dt_fixed = 5e-9
    to = 0.0
    for _ in range(10):
        nv.rk_step(ctx, U, T, t, dt_fixed, case.cfl, None, None)
        Uo, To, _ = oracle.rk.rk_step(mt, g, Uo, To, to, dt_fixed, None)
        to += dt_fixed
    nv.check(ctx)
    err = state_rel_l2(U, Uo, case.mech.n_species)
    assert err.max() < 1e-5, err


def test_fault_injection_is_reported_not_trapped():
    """Host-side injected NaN, a Newton cap of 0 and a negative density come back
    as status codes with the offending cell; the context stays usable."""
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case)
    out = torch.empty_like(U)
    bad = U.clone()
    bad[-1, 1234] = float("nan")
    nv.rhs(ctx, bad, T.clone(), 0.0, None, out)
    code, cell = nv.status(ctx)
    assert code in (nv.RF_ENONFINITE, nv.RF_ENEWTON) and cell == 1234
    nv.set_option(ctx, "newton_maxit", 0)
    nv.rhs(ctx, U, T.clone(), 0.0, None, out)
    code, cell = nv.status(ctx)
    assert code == nv.RF_ENEWTON and cell >= 0
    nv.set_option(ctx, "newton_maxit", 30)
    neg = U.clone()
    neg[:4, 77] = -neg[:4, 77]
    nv.rhs(ctx, neg, T.clone(), 0.0, None, out)
    code, cell = nv.status(ctx)
    assert code != nv.RF_OK and cell == 77
    nv.rhs(ctx, U, T, 0.0, None, out)                   # still usable
    assert nv.status(ctx)[0] == nv.RF_OK


def test_diagnostics_parity():
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case)
    d = nv.diagnostics(ctx, U, T)
    mt, g, Uo, To = oracle_setup(case)
    dV = g.dx * g.dy * g.dz
    Uf = Uo.reshape(Uo.shape[0], -1)
    tot = (Uf.sum(1) * dV).numpy()
    scale = (Uf.abs().sum(1) * dV).numpy()          # totals can cancel (momentum): compare to sum |U|
    assert np.all(np.abs(d["total"] - tot) <= 1e-13 * scale)
    st = oracle.rhs.primitives(mt, Uo, To)
    w = oracle.chemistry.production_rates(mt, st["rho_s"], st["T"])
    hrr = float(oracle.chemistry.heat_release_rate(mt, w, st["T"]).sum()) * dV
    assert abs(d["heat_release"] - hrr) <= 1e-12 * abs(hrr)
    # the maximum is exact, the temperatures themselves are Newton results (rounding level)
    assert abs(d["max_T"] - float(st["T"].max())) <= 1e-13 * float(st["T"].max())
