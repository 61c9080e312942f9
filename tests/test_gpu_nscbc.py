"""Characteristic (NSCBC) inflow and outflow boundaries (Application examples: the
diffusion flame's and the combustor's NSCBC boundaries) through the C ABI against
the FP64 oracle on the same seeded inputs: the FP64 RHS within 1e-12 per conserved
variable with WENO3-Z and TENO6, over subsonic and partly supersonic states, inflow
targets and outflow relaxation on every axis; FP64 RK steps likewise; the mixed
RHS within 1e-4 of each group's scale; the mixed state after a run of steps within
1e-5 (WENO3-Z) or within the oracle's own sensitivity (TENO6); batched ensembles with
NSCBC members match the member loop bitwise; the entry points that do not support
NSCBC reject it; and a longer injection run on the GPU alone holds the inflow plane
at its target."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02319_b300 import synth
from tests.gpu_common import (gpu_setup, laser_tuple, nscbc_oracle, oracle_setup, rel_inf, rel_inf_group,
                              state_rel_l2)
from tests.helpers import random_prim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
NO_LASER = {"laser": False}


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _target(g, mech, n_plane, prim, axis, side):
    """A random inflow target near the state of the boundary layer."""
    ns = mech.n_species
    lay = np.take(prim, 0 if side == 0 else prim.shape[3 - axis] - 1, axis=3 - axis)   # [5+ns, plane dims]
    lay = lay.reshape(5 + ns, -1)
    t = np.empty((4 + ns, n_plane))
    t[0:3] = lay[2:5] + g.uniform(-20.0, 20.0, (3, n_plane))
    t[3] = lay[1] * g.uniform(0.9, 1.1, n_plane)
    Y = lay[5:] * g.uniform(0.5, 1.5, (ns, n_plane))
    t[4:] = Y / Y.sum(0)
    return t


def _random_nscbc_case(shape, seed, vmax=50.0, axes=(0, 1, 2)):
    m = synth.mechanism_9sp(seed)
    nz, ny, nx = shape
    bc = [synth.BC_EXTRAPOLATE] * 3
    for a in axes:
        bc[a] = synth.BC_NSCBC
    grid = synth.Grid(nx, ny, nz, 1.1e-4, 0.9e-4, 1.3e-4, tuple(bc))
    prim = random_prim(m, shape, seed, smooth=True, vmax=vmax)
    g = np.random.default_rng(seed + 100)
    n3 = (nx, ny, nz)
    sides = {}
    for a in axes:
        n_plane = int(np.prod([n3[b] for b in range(3) if b != a]))
        for side in (0, 1):
            if (a + side) % 2 == 0:
                sides[(a, side)] = dict(p_inf=101325.0 * g.uniform(0.97, 1.03), sigma=float(g.uniform(0.0, 0.6)),
                                        target=None)
            else:
                sides[(a, side)] = dict(p_inf=101325.0, eta_u=float(g.uniform(0.2, 2.0)),
                                        eta_T=float(g.uniform(0.2, 2.0)), eta_t=float(g.uniform(0.2, 2.0)),
                                        eta_Y=float(g.uniform(0.2, 2.0)), length=float(g.uniform(0.0, 3e-3)),
                                        target=_target(g, m, n_plane, prim, a, side))
    return synth.Case(f"nscbc_random{shape}_v{int(vmax)}", m, grid, prim, synth.Laser(), nscbc=sides)


def _cases():
    return [synth.case_jet_inflow(0, 40, 24, 1),
            synth.case_jet_inflow(1, 20, 16, 12),
            _random_nscbc_case((7, 9, 13), 3),
            _random_nscbc_case((5, 6, 11), 4, vmax=700.0),
            _random_nscbc_case((4, 3, 130), 5, axes=(0,))]


CASES = _cases()


def _oracle_rhs(case, flags=None):
    mt, g, Uo, To = oracle_setup(case)
    fl = dict(flags or {}, nscbc=nscbc_oracle(case))
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, laser_tuple(case), fl)
    return ro


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_nscbc_rhs_parity_fp64(case, teno):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6 if teno else 0)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    ro = _oracle_rhs(case, {"scheme": "teno6"} if teno else None)
    err = rel_inf(out, ro)
    assert err.max() < TOL64, err


@pytest.mark.parametrize("flags", [1, 2, 4])
def test_nscbc_rhs_parity_term_switches(flags):
    """Inviscid part alone, inviscid off (no characteristic term either), chemistry off."""
    nv = _nv()
    case = CASES[2]
    mech, ctx, U, T = gpu_setup(case, flags=flags)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, None, out)
    nv.check(ctx)
    fl = {"inviscid": not (flags & 1), "viscous": not (flags & 2), "chemistry": not (flags & 4)}
    ro = _oracle_rhs(case, fl)
    assert rel_inf(out, ro).max() < TOL64


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
def test_nscbc_rhs_parity_mixed(teno):
    """FP32-bulk RHS on the 2-D injection case: per variable within 1e-4 of the
    oracle's largest value in its group (FP32 fluxes over 10^-4 m cells)."""
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED, flags=nv.RF_TENO6 if teno else 0)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, None, out)
    nv.check(ctx)
    ro = _oracle_rhs(case, {"scheme": "teno6"} if teno else None)
    err = rel_inf_group(out, ro, case.mech.n_species)
    assert err.max() < 1e-4, err


@pytest.mark.parametrize("case", [CASES[0], CASES[2]], ids=[CASES[0].name, CASES[2].name])
def test_nscbc_rk_step_parity_fp64(case):
    """Three FP64 steps at the CFL rule, the time step chosen by each side."""
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    fl = {"nscbc": nscbc_oracle(case)}
    to = 0.0
    for _ in range(3):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, None, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, None, 0.5, fl)
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf(U, Uo.reshape(U.shape)).max() < TOL64


def _oracle_run(case, U, T, fl, dt, steps):
    mt, g, _, _ = oracle_setup(case)
    for k in range(steps):
        U, T, _ = oracle.rk.rk_step(mt, g, U, T, k * dt, dt, None, 0.5, fl)
    return U


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
def test_nscbc_mixed_precision_state_error(teno):
    """Mixed path against the FP64 oracle after 30 steps of 20 ns of the 2-D
    injection case without the white noise (the inflow relaxation active over the
    jet), group-scaled relative L2.  WENO3-Z: within 1e-5.  TENO6: its keep / drop
    decisions near the inflow's sharp composition front make the oracle itself move
    by ~1e-3 when its initial state is perturbed by 1e-7 relative (FP32 rounding
    size), so the bar is three times that measured sensitivity; the RHS-level
    parity above holds TENO6's FP32 arithmetic to 1e-4 of each group's scale."""
    nv = _nv()
    case = synth.case_jet_inflow(0, 40, 24, 1, noise=0.0)
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED, flags=nv.RF_TENO6 if teno else 0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    fl = {"nscbc": nscbc_oracle(case)}
    if teno:
        fl["scheme"] = "teno6"
    dt = 2e-8
    for k in range(30):
        nv.rk_step(ctx, U, T, t, dt, 0.5, None, None)
    nv.check(ctx)
    ref = _oracle_run(case, Uo, To, fl, dt, 30)
    err = state_rel_l2(U, ref, case.mech.n_species)
    bar = 1e-5
    if teno:
        gen = torch.Generator().manual_seed(1)
        Up = Uo * (1.0 + 1e-7 * torch.randn(Uo.shape, generator=gen, dtype=torch.float64))
        sens = state_rel_l2(_oracle_run(case, Up, To, fl, dt, 30), ref, case.mech.n_species).max()
        bar = max(bar, 3.0 * float(sens))
    assert err.max() < bar, (err, bar)


def test_nscbc_injection_reaches_the_target():
    """The 3-D injection case on the GPU alone (FP64, 600 steps at CFL 0.5) with
    inflow relaxation coefficients of 20 (a nearly hard inflow; with 1 the jet's
    inflow velocity drifts far below its target while the interior accelerates, as
    partially reflecting inflows do): the state stays finite and the x-velocity of
    the inflow plane holds within 5 % of the target where the target is fastest."""
    nv = _nv()
    case = synth.case_jet_inflow(2, 48, 32, 32)
    case.nscbc[(0, 0)].update(eta_u=20.0, eta_T=20.0, eta_t=20.0, eta_Y=20.0)
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(600):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, None, None)
    nv.check(ctx)
    ns = case.mech.n_species
    g = case.grid
    Uv = U.reshape(ns + 4, g.nz, g.ny, g.nx)
    rho = Uv[:ns].sum(0)
    u_in = (Uv[ns] / rho)[:, :, 0].reshape(-1).cpu().numpy()
    tgt = case.nscbc[(0, 0)]["target"][0]
    k = int(np.argmax(tgt))
    assert abs(u_in[k] - tgt[k]) < 0.05 * tgt[k], (u_in[k], tgt[k])
    assert bool(torch.isfinite(U).all())


def test_nscbc_is_rejected_where_unsupported():
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    lam = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="NSCBC"):
        nv.adjoint_rhs(ctx, U, T, 0.0, None, lam, 0.0, lam.clone(), grads)
    with pytest.raises(RuntimeError, match="not an NSCBC axis"):
        nv.set_nscbc(ctx, 1, 0)
    with pytest.raises(RuntimeError, match=">= 0"):
        nv.set_nscbc(ctx, 0, 1, sigma=-1.0)
    with pytest.raises(RuntimeError, match="p_inf"):
        nv.set_nscbc(ctx, 0, 1, p_inf=0.0)
    small = synth.Grid(2, 8, 1, 1e-4, 1e-4, 1e-4, (synth.BC_NSCBC, synth.BC_PERIODIC, synth.BC_PERIODIC))
    with pytest.raises(RuntimeError, match="needs >= 3"):
        nv.create_ctx(mech, small, nv.RF_FP64)


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_nscbc_members_in_batched_ensembles_equal_the_member_loop(precision):
    """Members with characteristic ends (injection cases of uneven sizes, inflow
    targets of their own) beside a periodic member: every batched mode advances each
    member bitwise as the per-member loop does."""
    from tests.gpu_common import nscbc_gpu
    nv = _nv()
    cases = [synth.case_jet_inflow(3, 16, 12, 10), synth.case_jet_inflow(4, 12, 10, 8, u_jet=60.0),
             synth.ensemble_members(seed=2, n_members=1, lo=8, hi=12)[0]]
    res = {}
    for mode in (0, 1, 2, 3):
        mech = nv.init_mechanism(cases[0].mech)
        ctxs, Us, Ts = [], [], []
        for c in cases:
            ns, n = c.mech.n_species, c.grid.ncells
            ctx = nv.create_ctx(mech, c.grid, precision)
            U = torch.empty((ns + 4, n), dtype=torch.float64, device="cuda")
            T = torch.empty(n, dtype=torch.float64, device="cuda")
            nv.init_state(ctx, torch.as_tensor(c.prim, dtype=torch.float64).reshape(5 + ns, n).cuda(), U, T)
            nscbc_gpu(ctx, c)
            ctxs.append(ctx)
            Us.append(U)
            Ts.append(T)
        t = torch.zeros(len(cases), dtype=torch.float64, device="cuda")
        e = nv.ensemble_create(ctxs, Us, Ts, [c.laser.as_tuple() for c in cases], t)
        code, st = nv.run_ensemble(e, 3, mode, 0.5)
        assert code == 0 and st == [0] * len(cases)
        res[mode] = ([u.cpu() for u in Us], t.cpu())
        del e
    for mode in (1, 2, 3):
        for m in range(len(cases)):
            assert torch.equal(res[mode][0][m], res[0][0][m]), (mode, m)
        assert torch.equal(res[mode][1], res[0][1])
    assert float(res[0][1].min()) > 0.0
