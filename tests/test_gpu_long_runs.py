"""Long runs against the FP64 oracle on the same seeded inputs: the relative L2
state error after 100 (jet, ensemble) or 200 (mixing layer) fixed-dt SSP-RK3
steps.  Bar: mixed precision and the batched ensemble within 1e-5 (per conserved
variable, each scaled by its group's norm); the FP64 path within 1e-10 (rounding
growth over the run, from 1e-12 per RHS).

The fixed steps sit inside the time-step rule's limits over the whole run:
jet 1e-9 s against a chemical limit 0.2 / max|d omega / d rho| >= 0.95e-9 s after
the laser pulse (dt times the rate stays ~0.2, far inside RK3's linear stability
bound 2.5), mixing layer 5e-9 s against >= 6.6e-9 s."""
import pytest
import torch

import oracle
from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, laser_tuple, oracle_setup, state_rel_l2

pytestmark = pytest.mark.gpu


def _jet16():
    case = synth.case_jet(0, 16)
    case.laser.t0 = 5e-8            # the pulse (sigma_t = 10 ns) fires inside the run
    return case


def _oracle_run(case, dt, nsteps):
    mt, g, U, T = oracle_setup(case)
    las = laser_tuple(case)
    for k in range(nsteps):
        U, T, _ = oracle.rk.rk_step(mt, g, U, T, k * dt, dt, las)
    return U


def _gpu_run(case, precision, dt, nsteps):
    from paper_2202_02319_b300 import native as nv
    mech, ctx, U, T = gpu_setup(case, precision=precision)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(nsteps):
        nv.rk_step(ctx, U, T, t, dt, case.cfl, laser_tuple(case), None)
    nv.check(ctx)
    return U


@pytest.mark.parametrize("which", ["jet16_100", "mixing_layer64_200"])
def test_fp64_and_mixed_state_error_after_long_runs(which):
    from paper_2202_02319_b300 import native as nv
    if which == "jet16_100":
        case, dt, nsteps = _jet16(), 1e-9, 100
    else:
        case, dt, nsteps = synth.case_mixing_layer(0, 64), 5e-9, 200
    Uo = _oracle_run(case, dt, nsteps)
    ns = case.mech.n_species
    e64 = state_rel_l2(_gpu_run(case, nv.RF_FP64, dt, nsteps), Uo, ns)
    emx = state_rel_l2(_gpu_run(case, nv.RF_MIXED, dt, nsteps), Uo, ns)
    print(f"{which}: FP64 max rel L2 {e64.max():.3e}, mixed {emx.max():.3e}")
    assert e64.max() < 1e-10, e64
    assert emx.max() < 1e-5, emx


def test_ensemble_mixed_state_error_after_100_steps():
    """Three members of uneven size in one persistent launch per RK stage."""
    from paper_2202_02319_b300 import native as nv
    cases = synth.ensemble_members(seed=5, n_members=3, lo=8, hi=12, t0_max=1e-7)
    for c in cases:
        c.laser.E = 2e-3
        c.laser.t0 = 5e-8
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
    code, st = nv.run_ensemble(e, 100, nv.ENS_PERSISTENT, dt_fixed=1e-9)
    assert code == 0 and st == [0, 0, 0]
    for c, U in zip(cases, Us):
        err = state_rel_l2(U, _oracle_run(c, 1e-9, 100), c.mech.n_species)
        assert err.max() < 1e-5, (c.grid.nx, c.grid.ny, c.grid.nz, err)
