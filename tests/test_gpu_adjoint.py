"""The CUDA discrete adjoint: vector-Jacobian products of the RHS and of one RK
step against the oracle's reverse-mode derivatives (same seeded inputs), a
finite-difference dot-product check on the GPU, and the checkpointed ignition
gradient against central finite differences and the oracle's gradient."""
import numpy as np
import pytest
import torch

import oracle
from oracle import adjoint as oadj
from oracle.mech import from_synth, grid_from_synth
from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, oracle_setup

pytestmark = pytest.mark.gpu


def _case(n=8):
    case = synth.case_jet(0, n)
    dx = case.grid.dx
    case.laser.E = 2e-3
    case.laser.x0, case.laser.y0, case.laser.z0 = 3.9 * dx, 4.2 * dx, 3.7 * dx
    case.laser.sigma_r = 1.5 * dx
    case.laser.t0 = 1.5e-8
    return case


def _rel(a, b):
    a = a.reshape(a.shape[0], -1).double().cpu()
    b = b.reshape(b.shape[0], -1).double().cpu()
    return float(((a - b).abs().amax(1) / b.abs().amax(1).clamp_min(1e-300)).max())


def _oracle_vjp(case, lam, w_hrr, t):
    mt, g, Uo, To = oracle_setup(case)
    U = Uo.clone().requires_grad_(True)
    p = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in case.laser.as_tuple()[:5]]
    lnA = torch.log(mt.A.clone()).requires_grad_(True)
    m = mt.with_A(torch.exp(lnA))
    las = (p[0], p[1], p[2], p[3], p[4], case.laser.t0, case.laser.sigma_t)
    R, _ = oracle.rhs.rhs(m, g, U, To, t, las)
    H, _ = oadj.heat_release(m, g, U, To)
    obj = (R.reshape(R.shape[0], -1) * lam).sum() + w_hrr * H
    gr = torch.autograd.grad(obj, [U] + p + [lnA])
    return gr[0].reshape(R.shape[0], -1), torch.cat([torch.stack(gr[1:6]), gr[6]])


def test_adjoint_rhs_matches_oracle_reverse_mode():
    from paper_2202_02319_b300 import native as nv
    case = _case()
    mech, ctx, U, T = gpu_setup(case)
    g = torch.Generator().manual_seed(5)
    lam = torch.randn(U.shape, generator=g, dtype=torch.float64)
    t = case.laser.t0 - 3e-9
    w_hrr = 0.7
    lamU = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    nv.adjoint_rhs(ctx, U, T, t, case.laser.as_tuple(), lam.cuda(), w_hrr, lamU, grads)
    nv.check(ctx)
    gU, gp = _oracle_vjp(case, lam, w_hrr, t)
    assert _rel(lamU, gU) < 1e-10
    gpu = grads.cpu()
    assert float(((gpu - gp).abs() / gp.abs().clamp_min(1e-300 + gp.abs().max() * 1e-12)).max()) < 1e-9


def test_adjoint_rhs_without_inviscid_term_matches_oracle_to_rounding():
    from paper_2202_02319_b300 import native as nv
    case = _case()
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_NO_INVISCID)
    lam = torch.randn(U.shape, generator=torch.Generator().manual_seed(6), dtype=torch.float64)
    t = case.laser.t0 - 3e-9
    lamU = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    nv.adjoint_rhs(ctx, U, T, t, case.laser.as_tuple(), lam.cuda(), 0.3, lamU, grads)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    Ur = Uo.clone().requires_grad_(True)
    R, _ = oracle.rhs.rhs(mt, g, Ur, To, t, case.laser.as_tuple(), {"inviscid": False})
    H, _ = oadj.heat_release(mt, g, Ur, To)
    gU = torch.autograd.grad((R.reshape(R.shape[0], -1) * lam).sum() + 0.3 * H, [Ur])[0]
    assert _rel(lamU, gU.reshape(lamU.shape[0], -1)) < 1e-12


def test_adjoint_rhs_dot_product_with_finite_differences():
    """<lambda, (R(U + h w) - R(U - h w)) / 2h> = <J^T lambda, w> on the GPU."""
    from paper_2202_02319_b300 import native as nv
    case = _case()
    mech, ctx, U, T = gpu_setup(case)
    g = torch.Generator().manual_seed(7)
    lam = torch.randn(U.shape, generator=g, dtype=torch.float64).cuda()
    # relative perturbation of every entry: a sign change of a near-zero density would
    # cross the pole of the mixture-averaged diffusivity at X_s + eps = 0
    w = torch.randn(U.shape, generator=g, dtype=torch.float64).cuda() * U
    lamU = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    t = case.laser.t0
    nv.adjoint_rhs(ctx, U, T.clone(), t, case.laser.as_tuple(), lam, 0.0, lamU, grads)
    h = 1e-8              # small enough that no LLF maximum or |beta1 - beta0| kink is crossed
    Rp, Rm = torch.empty_like(U), torch.empty_like(U)
    nv.rhs(ctx, U + h * w, T.clone(), t, case.laser.as_tuple(), Rp)
    nv.rhs(ctx, U - h * w, T.clone(), t, case.laser.as_tuple(), Rm)
    nv.check(ctx)
    lhs = float((lam * (Rp - Rm)).sum()) / (2 * h)
    rhs_ = float((lamU * w).sum())
    assert abs(lhs - rhs_) <= 1e-6 * abs(rhs_)


def test_adjoint_rk_step_matches_oracle():
    from paper_2202_02319_b300 import native as nv
    case = _case()
    mech, ctx, U, T = gpu_setup(case)
    g = torch.Generator().manual_seed(9)
    lam1 = torch.randn(U.shape, generator=g, dtype=torch.float64)
    dt, t = 4e-9, case.laser.t0 - 8e-9
    lam = lam1.cuda().clone()
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    nv.adjoint_rk_step(ctx, U, T, t, dt, case.laser.as_tuple(), 1.0, lam, grads)
    nv.check(ctx)
    mt, gr, Uo, To = oracle_setup(case)
    Ur = Uo.clone().requires_grad_(True)
    p = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in case.laser.as_tuple()[:5]]
    lnA = torch.log(mt.A.clone()).requires_grad_(True)
    las = (p[0], p[1], p[2], p[3], p[4], case.laser.t0, case.laser.sigma_t)
    Un, _, dJ = oadj.step_objective(mt.with_A(torch.exp(lnA)), gr, Ur, To, t, dt, las)
    obj = (Un.reshape(Un.shape[0], -1) * lam1).sum() + dJ
    res = torch.autograd.grad(obj, [Ur] + p + [lnA])
    assert _rel(lam, res[0].reshape(lam.shape[0], -1)) < 1e-10
    gp = torch.cat([torch.stack(res[1:6]), res[6]])
    assert float(((grads.cpu() - gp).abs() / gp.abs().clamp_min(gp.abs().max() * 1e-12)).max()) < 1e-9


def test_checkpointed_gradient_vs_finite_differences_and_oracle():
    """dJ/dp of the time-integrated heat release over 12 steps (checkpoint every
    5) by the autograd.Function: matches central differences of the GPU forward
    (h = 1e-6 relative) to 1e-6 and the oracle's reverse-mode gradient to 1e-9."""
    from paper_2202_02319_b300 import adjoint
    case = _case()
    prob = adjoint.HeatReleaseProblem(case.mech, case.grid, case.prim, case.laser, nsteps=12, dt=4e-9,
                                      checkpoint_every=5)
    p0 = prob.default_params()
    p = p0.clone().requires_grad_(True)
    J = adjoint.ignition_objective(p, prob)
    J.backward()
    g = p.grad.clone()
    assert float(J) > 0.0
    # central differences of the GPU forward for the laser parameters and the three largest ln A
    check = [0, 1, 2, 3, 4] + [5 + int(j) for j in torch.argsort(g[5:].abs(), descending=True)[:3]]
    for i in check:
        h = 1e-6 * abs(float(p0[i])) if i < 5 else 1e-6
        pp, pm = p0.clone(), p0.clone()
        pp[i] += h
        pm[i] -= h
        fd = (prob.run(pp, keep=False) - prob.run(pm, keep=False)) / (2 * h)
        assert abs(fd - float(g[i])) <= 1e-6 * abs(fd) + 1e-9 * float(g.abs().max()), (i, fd, float(g[i]))
    # the oracle's gradient of the same objective
    mt, gr, Uo, To = oracle_setup(case)
    q = [torch.tensor(float(v), dtype=torch.float64, requires_grad=True) for v in p0[:5]]
    lnA = p0[5:].clone().requires_grad_(True)
    las = (q[0], q[1], q[2], q[3], q[4], case.laser.t0, case.laser.sigma_t)
    Jo = oadj.objective(mt, gr, Uo, To, 0.0, 4e-9, 12, las, lnA)
    res = torch.autograd.grad(Jo, q + [lnA])
    go = torch.cat([torch.stack(res[:5]), res[5]])
    assert abs(float(J) - float(Jo)) <= 1e-10 * abs(float(Jo))
    assert float(((g - go).abs() / go.abs().clamp_min(go.abs().max() * 1e-12)).max()) < 1e-8


def test_objective_nodes_keep_their_own_checkpoints():
    """Two differentiable runs of one problem before either backward: each graph node
    differentiates its own run (the checkpoints travel with the node), so the
    gradient of J(p1) taken after J(p2) was formed equals that of a lone J(p1)."""
    from paper_2202_02319_b300 import adjoint
    case = _case()
    prob = adjoint.HeatReleaseProblem(case.mech, case.grid, case.prim, case.laser, nsteps=6, dt=4e-9,
                                      checkpoint_every=4)
    p0 = prob.default_params()
    p1 = p0.clone()
    p1[0] *= 1.5
    a = p0.clone().requires_grad_(True)
    adjoint.ignition_objective(a, prob).backward()
    b0 = p0.clone().requires_grad_(True)
    b1 = p1.clone().requires_grad_(True)
    J0 = adjoint.ignition_objective(b0, prob)
    J1 = adjoint.ignition_objective(b1, prob)
    J0.backward()
    J1.backward()
    assert torch.allclose(b0.grad, a.grad, rtol=1e-9, atol=1e-12 * float(a.grad.abs().max()))
    assert not torch.allclose(b1.grad, a.grad, rtol=1e-6, atol=0.0)


def test_stored_stages_match_recomputation():
    """rf_rk_step_stages advances the state bit for bit as rf_rk_step_objective does,
    and the reverse step from its kept stage inputs (rf_adjoint_rk_step_stored) equals
    the recomputing one (rf_adjoint_rk_step) to the order of the FP64 atomic sums; the
    checkpointed gradient with and without stored stages likewise."""
    from paper_2202_02319_b300 import adjoint, native as nv
    case = _case()
    mech, ctx, U, T = gpu_setup(case)
    las = case.laser.as_tuple()
    dt, t = 4e-9, case.laser.t0 - 8e-9
    U0, T0 = U.clone(), T.clone()
    st = torch.empty(nv.stages_size(ctx), dtype=torch.float64, device="cuda")
    Ua, Ta = U.clone(), T.clone()
    Ja = nv.rk_step_stages(ctx, Ua, Ta, t, dt, las, st, want_J=True)
    Ub, Tb = U.clone(), T.clone()
    Jb = nv.rk_step_objective(ctx, Ub, Tb, t, dt, las)
    nv.check(ctx)
    assert torch.equal(Ua, Ub) and torch.equal(Ta, Tb) and Ja == Jb
    g = torch.Generator().manual_seed(11)
    lam0 = torch.randn(U.shape, generator=g, dtype=torch.float64).cuda()
    la, lb = lam0.clone(), lam0.clone()
    ga = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    gb = torch.zeros_like(ga)
    nv.adjoint_rk_step(ctx, U0, T0, t, dt, las, 1.0, la, ga)
    # stages of the plain step (no heat-release evaluation), as the gradient keeps them
    st2 = torch.empty_like(st)
    nv.rk_step_stages(ctx, U0.clone(), T0.clone(), t, dt, las, st2)
    nv.adjoint_rk_step_stored(ctx, U0, st2, t, dt, las, 1.0, lb, gb)
    nv.check(ctx)
    assert _rel(lb, la) < 1e-13
    assert float(((gb - ga).abs() / ga.abs().clamp_min(ga.abs().max() * 1e-12)).max()) < 1e-12
    with pytest.raises(ValueError):
        nv.rk_step_stages(ctx, U0.clone(), T0.clone(), t, dt, las, st[:10])
    grads = []
    for store in (True, False):
        prob = adjoint.HeatReleaseProblem(case.mech, case.grid, case.prim, case.laser, nsteps=7, dt=4e-9,
                                          checkpoint_every=4, store_stages=store)
        p = prob.default_params()
        J, state = prob.run_with_state(p)
        grads.append(prob.gradient(state))
    assert float(((grads[0] - grads[1]).abs() / grads[1].abs().clamp_min(grads[1].abs().max() * 1e-12)).max()) < 1e-11
