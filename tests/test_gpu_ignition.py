"""The minimum-ignition-energy search on the GPU (batched ensembles, FP64) gives
the oracle's bracket on the same seeded case: every member's ignited / failed
decision (peak T against 600 K, growth of the total heat release) agrees, and so
do the peak temperatures and heat release rates behind them."""
import pytest
import torch

from oracle import ignition as oig
from oracle.mech import from_synth, grid_from_synth
from paper_2202_02319_b300 import synth

pytestmark = pytest.mark.gpu


def _case():
    case = synth.case_jet(0, 8)
    dx = case.grid.dx
    case.laser.sigma_r = 1.5 * dx
    case.laser.t0 = 2e-8
    case.laser.x0 = case.laser.y0 = case.laser.z0 = 4 * dx
    return case


@pytest.mark.parametrize("mode", ["graph", "persistent"])
def test_minimum_ignition_energy_matches_the_oracle(mode):
    from paper_2202_02319_b300 import ignition, native as nv
    case = _case()
    members, rounds, nsteps, dt = 3, 2, 30, 2e-9
    runner = ignition.EnsembleIgnition(case, members, nsteps, dt, precision=nv.RF_FP64,
                                       mode=nv.ENS_GRAPH if mode == "graph" else nv.ENS_PERSISTENT)
    res = ignition.minimum_ignition_energy(runner, 0.02e-3, 3e-3, rounds=rounds)
    mt, g = from_synth(case.mech), grid_from_synth(case.grid)
    prim = torch.as_tensor(case.prim, dtype=torch.float64)
    (lo, hi), hist = oig.minimum_ignition_energy(mt, g, prim, case.laser.as_tuple(), 0.02e-3, 3e-3, members,
                                                 rounds, nsteps, dt)
    assert res.bracket == pytest.approx((lo, hi), rel=1e-14)
    assert any(any(r.ignited) for r in res.rounds) and any(not all(r.ignited) for r in res.rounds)
    for r, (probes, outcomes, _) in zip(res.rounds, hist):
        assert r.ignited == outcomes
        for E, mT, hm, he in zip(r.energies, r.max_T, r.hrr_mid, r.hrr_end):
            peak, h_mid, h_end = oig.member_window(mt, g, prim, (E,) + case.laser.as_tuple()[1:], nsteps, dt)
            assert abs(mT - peak) <= 1e-11 * peak
            assert abs(he - h_end) <= 1e-9 * abs(h_end) + 1e-20


def test_minimum_ignition_energy_with_characteristic_ends_matches_the_oracle():
    """The same search with NSCBC outflow ends on the jet's axis (the paper's
    diffusion-flame ensembles run between characteristic boundaries): bracket and
    every member decision equal the oracle's."""
    from paper_2202_02319_b300 import ignition, native as nv
    case = _case()
    case.grid.bc = (synth.BC_NSCBC, 0, 0)
    case.nscbc = {(0, 0): dict(p_inf=synth.P_ATM, sigma=0.25, target=None),
                  (0, 1): dict(p_inf=synth.P_ATM, sigma=0.25, target=None)}
    members, rounds, nsteps, dt = 3, 2, 30, 2e-9
    runner = ignition.EnsembleIgnition(case, members, nsteps, dt, precision=nv.RF_FP64, mode=nv.ENS_GRAPH)
    res = ignition.minimum_ignition_energy(runner, 0.02e-3, 3e-3, rounds=rounds)
    from oracle import nscbc
    mt, g = from_synth(case.mech), grid_from_synth(case.grid)
    prim = torch.as_tensor(case.prim, dtype=torch.float64)
    fl = {"nscbc": {0: {0: nscbc.Side(p_inf=synth.P_ATM, sigma=0.25), 1: nscbc.Side(p_inf=synth.P_ATM, sigma=0.25)}}}
    (lo, hi), hist = oig.minimum_ignition_energy(mt, g, prim, case.laser.as_tuple(), 0.02e-3, 3e-3, members,
                                                 rounds, nsteps, dt, flags=fl)
    assert res.bracket == pytest.approx((lo, hi), rel=1e-14)
    for r, (probes, outcomes, _) in zip(res.rounds, hist):
        assert r.ignited == outcomes
