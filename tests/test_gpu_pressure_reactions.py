"""Third-body and fall-off (Lindemann, Troe) reactions through the C ABI
against the FP64 oracle on the same seeded inputs (the paper's CH4/O2
mechanisms contain such reactions; Methods - Combustion chemistry): FP64 RHS
within 1e-12 per conserved variable, the diagnostics' heat release, an FP64 RK
step with the time-step rule, and the mixed path within the 1e-5 state bar
after a run of steps; the adjoint, built for elementary reactions, rejects them."""
import pytest
import torch

import oracle
from oracle import adjoint as oadj
from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, laser_tuple, oracle_setup, rel_inf, state_rel_l2
from tests.helpers import random_prim

pytestmark = pytest.mark.gpu


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _cases():
    m = synth.mechanism_9sp_pressure(0)
    hot = synth.Case("hot_random", m, synth.Grid(13, 7, 5, 1.1e-4, 0.9e-4, 1.3e-4, (1, 0, 1)),
                     random_prim(m, (5, 7, 13), 3, T_lo=900.0, T_hi=2600.0))
    smooth = synth.Case("hot_smooth", m, synth.Grid(40, 6, 4, 1e-4, 1e-4, 1e-4, (0, 0, 0)),
                        random_prim(m, (4, 6, 40), 8, T_lo=1100.0, T_hi=2400.0, smooth=True))
    jet = synth.case_jet(0, 16)
    jet.mech = m
    jet.laser.t0 = 2e-8
    jet.laser.x0, jet.laser.y0, jet.laser.z0 = 8.3 * jet.grid.dx, 7.6 * jet.grid.dx, 8.1 * jet.grid.dx
    mix = synth.case_mixing_layer(0, 32)
    mix.mech = m
    return [hot, smooth, jet, mix]


CASES = _cases()


@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_pressure_reactions_rhs_parity_fp64(case):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case)
    out = torch.empty_like(U)
    las = laser_tuple(case)
    nv.rhs(ctx, U, T, 0.0, las, out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, las)
    assert rel_inf(out, ro).max() < 1e-12


def test_pressure_reactions_heat_release_and_step():
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case)
    d = nv.diagnostics(ctx, U, T.clone())
    mt, g, Uo, To = oracle_setup(case)
    H, _ = oadj.heat_release(mt, g, Uo, To)
    assert abs(d["heat_release"] - float(H)) <= 1e-12 * abs(float(H))
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    nv.rk_step(ctx, U, T, t, 0.0, 0.5, None, dt)
    nv.check(ctx)
    Uo2, _, dto = oracle.rk.rk_step(mt, g, Uo, To, 0.0, 0.0, None, 0.5)
    assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf(U, Uo2.reshape(U.shape)).max() < 1e-12


def test_pressure_reactions_mixed_state_error():
    """Mixed path on the 16^3 jet (pulse inside the run) with the pressure-dependent
    mechanism: group-scaled relative L2 within 1e-5 after 30 steps of 1 ns."""
    nv = _nv()
    case = CASES[2]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED)
    las = laser_tuple(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    for k in range(30):
        nv.rk_step(ctx, U, T, t, 1e-9, 0.5, las, None)
        Uo, To, _ = oracle.rk.rk_step(mt, g, Uo, To, k * 1e-9, 1e-9, las)
    nv.check(ctx)
    assert state_rel_l2(U, Uo, case.mech.n_species).max() < 1e-5


def test_adjoint_rejects_pressure_dependent_reactions():
    nv = _nv()
    case = CASES[2]
    mech, ctx, U, T = gpu_setup(case)
    lam = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="elementary"):
        nv.adjoint_rhs(ctx, U, T, 0.0, case.laser.as_tuple(), lam, 0.0, lam.clone(), grads)
