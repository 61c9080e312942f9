"""Pin of the oracle's gradient machinery: reverse-mode derivatives of the
heat-release objective agree with central finite differences of the same
objective (laser energy, position, width and ln A)."""
import numpy as np
import torch

from oracle import adjoint, rhs
from oracle.mech import from_synth, grid_from_synth
from paper_2202_02319_b300 import synth


def test_oracle_objective_gradient_matches_central_differences():
    case = synth.case_jet(0, 6)
    mt, g = from_synth(case.mech), grid_from_synth(case.grid)
    U0, T0 = rhs.init_state(mt, torch.as_tensor(case.prim, dtype=torch.float64))
    dx = case.grid.dx
    base = [2e-3, 2.9 * dx, 3.2 * dx, 2.7 * dx, 1.5 * dx]
    t0, st = 1.5e-8, 1e-8
    lnA0 = torch.log(mt.A.clone())
    dt, nsteps = 4e-9, 3

    def J_of(p, lnA):
        las = (p[0], p[1], p[2], p[3], p[4], t0, st)
        return adjoint.objective(mt, g, U0, T0, 0.0, dt, nsteps, las, lnA)
    p = [torch.tensor(v, dtype=torch.float64, requires_grad=True) for v in base]
    lnA = lnA0.clone().requires_grad_(True)
    J = J_of(p, lnA)
    grads = torch.autograd.grad(J, p + [lnA])
    gp = [float(x) for x in grads[:5]]
    gA = grads[5]
    for i in range(5):
        h = 1e-6 * abs(base[i])
        pp = [torch.tensor(v, dtype=torch.float64) for v in base]
        pm = [torch.tensor(v, dtype=torch.float64) for v in base]
        pp[i] = pp[i] + h
        pm[i] = pm[i] - h
        fd = (float(J_of(pp, lnA0)) - float(J_of(pm, lnA0))) / (2 * h)
        assert abs(fd - gp[i]) <= 1e-5 * max(abs(fd), 1e-12 * abs(float(J)) / h), (i, fd, gp[i])
    j = int(torch.argmax(gA.abs()))
    h = 1e-6
    ap, am = lnA0.clone(), lnA0.clone()
    ap[j] += h
    am[j] -= h
    fd = (float(J_of(base, ap)) - float(J_of(base, am))) / (2 * h)
    assert abs(fd - float(gA[j])) <= 1e-5 * abs(fd)
