"""TENO6 (the paper's sixth-order scheme; Results, Solver; Methods, Numerical
method) through the C ABI against the FP64 oracle on the same seeded inputs: the
FP64 RHS within 1e-12 per conserved variable, an FP64 RK step likewise, the
mixed path within the 1e-5 state bar after a run of steps; and the entry points
that do not support TENO6 reject it."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, laser_tuple, oracle_setup, rel_inf, state_rel_l2
from tests.helpers import random_prim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _random_case(shape, bc, seed, smooth=False):
    m = synth.mechanism_9sp(seed)
    nz, ny, nx = shape
    grid = synth.Grid(nx, ny, nz, 1.1e-4, 0.9e-4, 1.3e-4, bc)
    return synth.Case(f"random{shape}", m, grid, random_prim(m, shape, seed, smooth=smooth))


def _cases():
    jet = synth.case_jet(0, 16)
    jet.laser.t0 = 2e-8
    jet.laser.x0, jet.laser.y0, jet.laser.z0 = 8.3 * jet.grid.dx, 7.6 * jet.grid.dx, 8.1 * jet.grid.dx
    return [synth.case_box32(0), jet, synth.case_mixing_layer(0, 32),
            _random_case((5, 7, 13), (1, 0, 1), 3), _random_case((6, 5, 1), (0, 0, 0), 4),
            _random_case((1, 1, 1), (0, 0, 0), 5), _random_case((2, 3, 300), (0, 1, 0), 6, smooth=True),
            _random_case((4, 5, 257), (0, 0, 1), 8, smooth=True)]


CASES = _cases()
TENO = {"scheme": "teno6"}


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_teno6_rhs_parity_fp64(case):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6)
    out = torch.empty_like(U)
    las = laser_tuple(case)
    nv.rhs(ctx, U, T, 0.0, las, out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, las, TENO)
    err = rel_inf(out, ro)
    assert err.max() < TOL64, err


@pytest.mark.parametrize("flags", [1, 2])
def test_teno6_rhs_parity_term_switches(flags):
    """Inviscid part alone (viscous off) and viscous part alone with TENO6 set."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6 | flags)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    fl = {"scheme": "teno6", "inviscid": not (flags & 1), "viscous": not (flags & 2)}
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, laser_tuple(case), fl)
    assert rel_inf(out, ro).max() < TOL64


def test_teno6_rk_step_parity_fp64():
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6)
    las = laser_tuple(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    to = 0.0
    for _ in range(2):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, las, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, las, 0.5, TENO)
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf(U, Uo.reshape(U.shape)).max() < TOL64


def test_teno6_mixed_precision_state_error():
    """Mixed path (FP32 bulk, TENO6 in FP32) against the FP64 oracle after 20 steps of
    the 16^3 jet with the laser on: group-scaled relative L2 within 1e-5."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED, flags=nv.RF_TENO6)
    las = laser_tuple(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    dt = 2e-9
    for k in range(20):
        nv.rk_step(ctx, U, T, t, dt, 0.5, las, None)
        Uo, To, _ = oracle.rk.rk_step(mt, g, Uo, To, k * dt, dt, las, 0.5, TENO)
    nv.check(ctx)
    err = state_rel_l2(U, Uo, case.mech.n_species)
    assert err.max() < 1e-5, err


def test_teno6_is_rejected_where_unsupported():
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="TENO6"):
        nv.ensemble_create([ctx], [U], [T], [case.laser.as_tuple()], t)
    lam = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="TENO6"):
        nv.adjoint_rhs(ctx, U, T, 0.0, case.laser.as_tuple(), lam, 0.0, lam.clone(), grads)
    with pytest.raises(RuntimeError):
        nv.create_ctx(mech, case.grid, nv.RF_FP64, 128)          # no such flag bit
