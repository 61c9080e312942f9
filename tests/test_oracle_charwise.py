"""Pins of the oracle's characteristic-wise splitting (Methods, Numerical method:
the optional characteristic variant of the WENO3-Z / TENO6 flux splitting), each
against something outside the splitting code: the flux Jacobian of the oracle's
Euler flux by finite differences (eigenvalues and right eigenvectors), the oracle's
frozen sound speed, the exact invariants of the scheme (uniform state,
conservation), the Sod tube's exact solution and the vortex's convergence order."""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import charwise, fluxes, rhs, rk
from oracle.mech import GridT
from tests import cases_accuracy as ca
from tests import riemann_exact as rx
from tests.helpers import mech_t, random_prim, tensor


@pytest.fixture(scope="module")
def mech():
    return mech_t(synth.mechanism_4sp(0))


def _states(mt, n, seed):
    m = synth.mechanism_4sp(0)
    prim = tensor(random_prim(m, (1, 1, n), seed, vmax=200.0))
    U, T = rhs.init_state(mt, prim)
    st = rhs.primitives(mt, U, T)
    return U, T, st


@pytest.mark.parametrize("d", [0, 1, 2])
def test_eigenvectors_of_the_flux_jacobian(mech, d):
    """A R = R Lambda for dF_d/dU of the oracle's Euler flux (central differences
    through the conserved -> primitive map), Lambda = (u - c, u x (Ns + 2), u + c);
    and the closure c^2 = sum Y phi + b (H - |u|^2) is the frozen sound speed."""
    U, T, st = _states(mech, 6, 3 + d)
    ns = mech.ns
    b, phi, H = charwise.cell_quantities(mech, U, st["vel"], st["p"], st["c"], st["T"])
    ke2 = st["vel"][0] ** 2 + st["vel"][1] ** 2 + st["vel"][2] ** 2
    c2 = (st["Y"] * phi).sum(0) + b * (H - ke2)
    assert float(((c2 - st["c"] ** 2).abs() / st["c"] ** 2).max()) < 1e-12
    Rm = charwise.right_eigenvectors(st["Y"], st["vel"], phi, b, H, st["c"], d)   # [1, 1, n, nv, nv]

    def F(V):
        s2 = rhs.primitives(mech, V, st["T"])
        return fluxes.euler_flux(V, s2["vel"], s2["p"], d, ns)
    nv = ns + 4
    lam = torch.stack([st["vel"][d] - st["c"]] + [st["vel"][d]] * (ns + 2) + [st["vel"][d] + st["c"]])
    # each row's scale: its largest entry over all eigenvectors times the largest speed
    row_scale = Rm.abs().amax(dim=(0, 1, 2, 4))[:, None, None, None] * lam.abs().max()
    for col in range(nv):
        r = Rm[..., :, col].permute(3, 0, 1, 2)                  # [nv, 1, 1, n]
        eps = 1e-7 * U.abs().amax(dim=(1, 2, 3), keepdim=True).max() / r.abs().max()
        Ar = (F(U + eps * r) - F(U - eps * r)) / (2 * eps)
        want = lam[col][None] * r
        assert float(((Ar - want).abs() / row_scale).max()) < 1e-5, col


def test_uniform_state_and_conservation(mech):
    """Characteristic-wise splitting keeps a uniform state exactly and telescopes on
    a periodic box, with WENO3-Z and TENO6."""
    m = synth.mechanism_4sp(0)
    for scheme in ("weno3z", "teno6"):
        fl = {"splitting": "characteristic", "scheme": scheme, "chemistry": False, "laser": False}
        prim = tensor(random_prim(m, (5, 6, 7), 4, smooth=True))
        U, T = rhs.init_state(mech, prim)
        g = GridT(7, 6, 5, 1e-4, 1.2e-4, 0.9e-4, (0, 0, 0))
        R, _ = rhs.rhs(mech, g, U, T, flags=fl)
        tot = R.reshape(R.shape[0], -1).sum(1)
        mag = R.reshape(R.shape[0], -1).abs().sum(1)
        assert float((tot.abs() / mag).max()) < 1e-12
        uni = prim.clone()
        for k in range(prim.shape[0]):
            uni[k] = prim[k].mean()
        U, T = rhs.init_state(mech, uni)
        R, _ = rhs.rhs(mech, g, U, T, flags=fl)
        assert float(R.abs().max()) < 1e-6 * float(U.abs().max())


def test_sod_shock_tube_characteristic(mech):
    """Sod (Toro test 1) with characteristic-wise WENO3-Z: star-region pressure and
    velocity within 1 % and a density L1 error no larger than the component-wise
    scheme's, at N = 400."""
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sod_toro_test1.json")))
    g = gold["gamma"]
    L = (gold["left"]["rho"], gold["left"]["u"], gold["left"]["p"])
    Rt = (gold["right"]["rho"], gold["right"]["u"], gold["right"]["p"])
    ps, us = rx.star_state(L, Rt, g)
    mt = mech_t(ca.gas())
    n = 400
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    left = x < 0.5
    rho0 = np.where(left, L[0], Rt[0])
    p0 = np.where(left, L[2], Rt[2])
    prim = np.zeros((6, 1, 1, n))
    prim[0] = p0
    prim[1] = p0 / rho0
    prim[5] = 1.0
    res = {}
    for split in ("component", "characteristic"):
        U, T = rhs.init_state(mt, tensor(prim))
        grid = GridT(n, 1, 1, h, h, h, (1, 0, 0))
        fl = {"viscous": False, "chemistry": False, "laser": False, "splitting": split}
        t = 0.0
        while t < 0.2 - 1e-14:
            dt = min(rk.time_step(mt, grid, U, T, t, None, 0.5, fl), 0.2 - t)
            U, T, _ = rk.rk_step(mt, grid, U, T, t, dt, None, flags=fl)
            t += dt
        rho = U[0, 0, 0].numpy()
        ex = rx.sample(L, Rt, g, (x - 0.5) / t)
        res[split] = (np.abs(rho - ex[0]).mean(), U, T)
    U, T = res["characteristic"][1], res["characteristic"][2]
    st = rhs.primitives(mt, U, T)
    p = st["p"][0, 0].numpy()
    u = (U[1, 0, 0] / U[0, 0, 0]).numpy()
    xs = 0.5 + rx.shock_speed_right(L, Rt, g) * 0.2
    band = (x > 0.5 + us * 0.2 + 0.03) & (x < xs - 0.02)
    assert abs(p[band].mean() - ps) < 0.01 * ps
    assert abs(u[band].mean() - us) < 0.01 * us
    assert res["characteristic"][0] <= 1.05 * res["component"][0]


def test_vortex_converges_at_third_order_characteristic():
    """The isentropic vortex (Cartesian, t = 0.05) with characteristic-wise WENO3-Z:
    third order between N = 64 and 128."""
    mt = mech_t(ca.gas())
    errs = []
    for N in (32, 64, 128):
        prim, _, dx = ca.vortex_prim(N)
        g = GridT(N, N, 1, dx, dx, dx)
        U, T = rhs.init_state(mt, tensor(prim))
        t, dt = 0.0, 1e-3
        fl = {"viscous": False, "chemistry": False, "laser": False, "splitting": "characteristic"}
        for _ in range(50):
            U, T, _ = rk.rk_step(mt, g, U, T, t, dt, None, flags=fl)
            t += dt
        _, rex, _ = ca.vortex_prim(N, t)
        errs.append(np.abs(U[0, 0].numpy() - rex).mean())
    assert math.log2(errs[1] / errs[2]) > 2.7, errs
