"""Ignition sensitivities by the discrete adjoint (RK-step checkpointing plus
recomputation), behind a torch.autograd.Function.

Objective (the ignition measure of the paper's sensitivity question,
Application examples): the time-integrated heat release of a run of fixed-dt
SSP-RK3 steps, J = sum_n dt sum_k b_k H(U^(k)), b = (1/6, 1/6, 2/3) over the
stage inputs, H = sum over cells of -sum_s h_s omega_s times the cell volume.
Parameters p = (E, x0, y0, z0, sigma_r, ln A_0 .. ln A_{Nr-1}).

The forward run keeps the state every `checkpoint_every` steps; the reverse run
restores each checkpoint, recomputes the states of its segment and walks back
through them with rf_adjoint_rk_step.  With store_stages (the default) the
recomputation also keeps each step's stage inputs (rf_rk_step_stages, (2 (Ns + 4)
+ 3) N doubles per step of a segment), so that the reverse of every step but the
segment's last skips the two RHS evaluations that recompute them
(rf_adjoint_rk_step_stored).  All arithmetic is in the CUDA library; this module
only schedules calls and stores states.
"""
from __future__ import annotations

import copy

import numpy as np
import torch

from . import native as nv


class HeatReleaseProblem:
    def __init__(self, mech, grid, prim, laser, nsteps: int, dt: float, t0: float = 0.0,
                 checkpoint_every: int = 20, device="cuda", store_stages: bool = True):
        self.mech0 = mech
        self.grid = grid
        self.prim = torch.as_tensor(prim, dtype=torch.float64).reshape(5 + mech.n_species, -1)
        self.laser = laser
        self.nsteps = int(nsteps)
        self.dt = float(dt)
        self.t0 = float(t0)
        self.ck = max(1, int(checkpoint_every))
        self.store_stages = bool(store_stages)
        self.device = torch.device(device)
        self.np = 5 + mech.n_reactions
        self._state = None

    def default_params(self) -> torch.Tensor:
        l = self.laser
        return torch.tensor([l.E, l.x0, l.y0, l.z0, l.sigma_r] + list(np.log(self.mech0.A)), dtype=torch.float64)

    def _setup(self, params):
        p = params.detach().cpu().double().numpy()
        m = copy.deepcopy(self.mech0)
        m.A = np.exp(p[5:])
        las = (p[0], p[1], p[2], p[3], p[4], self.laser.t0, self.laser.sigma_t)
        mech = nv.init_mechanism(m)
        ctx = nv.create_ctx(mech, self.grid, nv.RF_FP64)
        n = self.grid.ncells
        U = torch.empty((m.n_species + 4, n), dtype=torch.float64, device=self.device)
        T = torch.empty(n, dtype=torch.float64, device=self.device)
        nv.init_state(ctx, self.prim.to(self.device), U, T)
        return mech, ctx, U, T, las

    def run_with_state(self, params):
        """J(p) and the run's reverse-sweep state (handles and checkpoints), which
        gradient() takes; each call owns its state, so several runs can be
        differentiated in any order."""
        mech, ctx, U, T, las = self._setup(params)
        J = 0.0
        cks = {}
        for k in range(self.nsteps):
            if k % self.ck == 0:
                cks[k] = (U.clone(), T.clone())
            J += nv.rk_step_objective(ctx, U, T, self.t0 + k * self.dt, self.dt, las)
        nv.check(ctx)
        return J, (mech, ctx, las, cks)

    def run(self, params, keep: bool = True) -> float:
        """J(p); with keep, the run's state is also kept as the default of gradient()."""
        if keep:
            J, self._state = self.run_with_state(params)
            return J
        mech, ctx, U, T, las = self._setup(params)
        J = 0.0
        for k in range(self.nsteps):
            J += nv.rk_step_objective(ctx, U, T, self.t0 + k * self.dt, self.dt, las)
        nv.check(ctx)
        return J

    def gradient(self, state=None) -> torch.Tensor:
        """dJ/dp of the run that produced `state` (default: the last run(keep=True)),
        by the reverse sweep."""
        mech, ctx, las, cks = state if state is not None else self._state
        lam = torch.zeros((mech.n_species + 4, self.grid.ncells), dtype=torch.float64, device=self.device)
        grads = torch.zeros(self.np, dtype=torch.float64, device=self.device)
        for k0 in sorted(cks, reverse=True):
            k1 = min(k0 + self.ck, self.nsteps)
            U, T = cks[k0][0].clone(), cks[k0][1].clone()
            seg = []
            for k in range(k0, k1):                # recompute the segment's step inputs
                if k + 1 < k1 and self.store_stages:
                    # keep the step's stage inputs: its reverse then skips two RHS
                    st = torch.empty(nv.stages_size(ctx), dtype=torch.float64, device=self.device)
                    seg.append((U.clone(), None, st))
                    nv.rk_step_stages(ctx, U, T, self.t0 + k * self.dt, self.dt, las, st)
                else:
                    seg.append((U.clone(), T.clone(), None))
                    if k + 1 < k1:
                        nv.rk_step_objective(ctx, U, T, self.t0 + k * self.dt, self.dt, las, want_J=False)
            for k in range(k1 - 1, k0 - 1, -1):
                Un, Tn, st = seg[k - k0]
                if st is not None:
                    nv.adjoint_rk_step_stored(ctx, Un, st, self.t0 + k * self.dt, self.dt, las, 1.0, lam, grads)
                else:
                    nv.adjoint_rk_step(ctx, Un, Tn, self.t0 + k * self.dt, self.dt, las, 1.0, lam, grads)
                seg[k - k0] = None
        nv.check(ctx)
        return grads.cpu()


class _Objective(torch.autograd.Function):
    @staticmethod
    def forward(fctx, params, problem):
        # the checkpoints of this run travel with this graph node, so a later run of
        # the same problem does not change this node's gradient
        J, fctx.state = problem.run_with_state(params)
        fctx.problem = problem
        return params.new_tensor(J)

    @staticmethod
    def backward(fctx, gJ):
        g = fctx.problem.gradient(fctx.state)
        fctx.state = None
        return gJ * g.to(gJ.device, gJ.dtype), None


def ignition_objective(params: torch.Tensor, problem: HeatReleaseProblem) -> torch.Tensor:
    """Differentiable J(p): forward by the CUDA path, gradient by its discrete adjoint."""
    return _Objective.apply(params, problem)
