"""Pins of the oracle's flux divergence: exact invariants (uniform state,
telescoping conservation, axis symmetry), closed-form discrete diffusion
operators, the Sod shock tube against the exact Riemann solution, and the
paper's accuracy problems (Methods, Solver Performance Analysis, Accuracy)."""
import json
import math
import os

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import fluxes, rhs, rk, thermo, transport
from oracle.mech import GridT
from tests import cases_accuracy as ca
from tests import riemann_exact as rx
from tests.helpers import mech_t, random_prim, single_species, tensor, R

NOSRC = {"chemistry": False, "laser": False}


def test_uniform_state_is_preserved():
    m = synth.mechanism_9sp(0)
    mt = mech_t(m)
    g = np.random.default_rng(0)
    Y = g.dirichlet(np.ones(9))
    vals = np.concatenate([[1.3e5, 900.0, 37.0, -12.0, 5.0], Y])
    prim = vals.reshape(-1, 1, 1, 1) * np.ones((1, 5, 6, 7))
    U, T = rhs.init_state(mt, tensor(prim))
    grid = GridT(7, 6, 5, 1e-4, 2e-4, 1.5e-4)
    out, _, st = rhs.rhs(mt, grid, U, T, 0.0, None, NOSRC, return_state=True)
    # Torch's vectorised transcendental functions round differently in SIMD lanes
    # and scalar tails, so cells agree to an ulp rather than bitwise; measure the
    # residual against the size of the individual face-flux terms alpha |U| / h.
    alpha = float((st["vel"][0].abs() + st["c"]).max()) + 40.0
    scale = alpha * U.abs().amax(dim=(1, 2, 3)) / 1e-4
    assert float((out.abs().amax(dim=(1, 2, 3)) / scale).max()) < 1e-12


@pytest.mark.parametrize("mk", [synth.mechanism_4sp, synth.mechanism_9sp])
def test_periodic_telescoping_conservation(mk):
    """sum over cells of every RHS component vanishes on a periodic box (species
    mass, momentum, energy) when the sources are off."""
    m = mk(0)
    mt = mech_t(m)
    prim = random_prim(m, (6, 7, 8), 3, vmax=80.0)
    U, T = rhs.init_state(mt, tensor(prim))
    grid = GridT(8, 7, 6, 1e-4, 1.2e-4, 0.9e-4)
    out, _ = rhs.rhs(mt, grid, U, T, 0.0, None, NOSRC)
    tot = out.sum(dim=(1, 2, 3))
    scale = out.abs().sum(dim=(1, 2, 3))
    assert float((tot.abs() / scale).max()) < 1e-13


def test_axis_permutation_symmetry():
    """Rotating the field x->y->z->x (and the velocity components with it) rotates
    the RHS."""
    m = synth.mechanism_9sp(1)
    mt = mech_t(m)
    n = 6
    prim = random_prim(m, (n, n, n), 5, smooth=True)
    U, T = rhs.init_state(mt, tensor(prim))
    grid = GridT(n, n, n, 1e-4, 1e-4, 1e-4)
    out, _ = rhs.rhs(mt, grid, U, T, 0.0, None, NOSRC)
    ns = 9

    def rot(V):
        # new field f'(z, y, x) = f(y, x, z): axes (z, y, x) -> tensor permute (y, x, z)
        W = V.permute(0, 2, 3, 1).clone()
        mom = W[ns:ns + 3].clone()
        W[ns + 0], W[ns + 1], W[ns + 2] = mom[2], mom[0], mom[1]
        return W
    U2 = rot(U)
    T2 = T.permute(1, 2, 0).clone()
    out2, _ = rhs.rhs(mt, grid, U2, T2, 0.0, None, NOSRC)
    ref = rot(out)
    err = (out2 - ref).abs().amax(dim=(1, 2, 3)) / ref.abs().amax(dim=(1, 2, 3))
    assert float(err.max()) < 1e-12


def test_weno3z_reconstruction_is_third_order_on_monotone_data():
    """Away from critical points WENO3-Z is third order: in the conservative
    finite-difference form the point values f_i are cell averages of a function
    g with g(x_{i+1/2}) = f(x_{i+1/2}) - h^2/24 f''(x_{i+1/2}) + O(h^4), and the
    reconstruction at i+1/2 (and its mirror from the right) meets g to O(h^3)."""
    errs = []
    for n in (40, 80, 160):
        h = 1.0 / n
        x = np.arange(-2, n + 2) * h
        f = torch.tensor(np.exp(x) + x, dtype=torch.float64)
        got = fluxes.weno3z(f[1:-3], f[2:-2], f[3:-1], h)       # faces (i+1/2), i = 2..n+1
        xf = x[2:-2] + h / 2
        exact = np.exp(xf) + xf - h * h / 24.0 * np.exp(xf)
        mirror = fluxes.weno3z(f[4:], f[3:-1], f[2:-2], h)       # from the right, same faces
        errs.append((np.abs(got.numpy() - exact).max(), np.abs(mirror.numpy() - exact).max()))
    for k in range(2):
        for a, b in zip(errs[:-1], errs[1:]):
            assert math.log2(a[k] / b[k]) > 2.8


def test_weno3z_keeps_third_order_at_a_smooth_extremum():
    """At a smooth extremum (f' = 0) the grid-scaled eps keeps WENO3-Z third order:
    f = cos(pi x) around x = 0 is the cell average of g = f (pi h / 2) / sin(pi h / 2),
    and the reconstruction at the faces within 0.1 of the extremum meets g to O(h^3)."""
    errs = []
    for n in (80, 160, 320):
        h = 1.0 / n
        x = (np.arange(-2, n + 2) - n / 2 + 0.25) * h
        f = torch.tensor(np.cos(np.pi * x), dtype=torch.float64)
        got = fluxes.weno3z(f[1:-3], f[2:-2], f[3:-1], h).numpy()
        xf = x[2:-2] + h / 2
        exact = np.cos(np.pi * xf) * (np.pi * h / 2) / np.sin(np.pi * h / 2)
        near = np.abs(xf) < 0.1
        errs.append(np.abs(got - exact)[near].max())
    for a, b in zip(errs[:-1], errs[1:]):
        assert math.log2(a / b) > 2.8


def test_linear_diffusion_operators_closed_form():
    """At rest, uniform p: (i) a small temperature sine gives an energy RHS of
    lambda(T0) times the discrete Laplacian eigenvalue -4 sin^2(k h / 2) / h^2;
    (ii) a shear sine u(y) gives mu times the same; (iii) a compression sine u(x)
    gives (4/3) mu times it."""
    W = 0.029
    m = single_species(gamma=1.4, W=W, mu=2e-5, mu_exp=0.7)
    mt = mech_t(m)
    n, h = 32, 1e-3
    k = 2 * math.pi * 3 / (n * h)
    x = (np.arange(n) + 0.5) * h
    eig = -4.0 * math.sin(k * h / 2) ** 2 / h ** 2
    T0, dT = 400.0, 1e-4
    cp = 3.5 * R / W
    mu0 = 2e-5 * (T0 / 300.0) ** 0.7
    lam0 = mu0 * (cp + 1.25 * R / W)
    fl = {"inviscid": False, "chemistry": False, "laser": False}
    # (i) heat conduction along x
    prim = np.zeros((6, 1, 1, n))
    prim[0] = 1e5
    prim[1] = T0 + dT * np.sin(k * x)
    prim[5] = 1.0
    U, T = rhs.init_state(mt, tensor(prim))
    out, _ = rhs.rhs(mt, GridT(n, 1, 1, h, h, h), U, T, 0.0, None, fl)
    np.testing.assert_allclose(out[4, 0, 0].numpy(), lam0 * eig * dT * np.sin(k * x), rtol=2e-6, atol=1e-12 * lam0 * abs(eig) * dT)
    assert float(out[0].abs().max()) == 0.0
    # (ii) shear wave u(y), (iii) compression wave u(x)
    du = 1e-3
    for axis, factor in (("y", 1.0), ("x", 4.0 / 3.0)):
        prim = np.zeros((6, 1, n, n))
        prim[0] = 1e5
        prim[1] = T0
        prim[5] = 1.0
        coord = x[:, None] if axis == "y" else x[None, :]
        prim[2] = du * np.sin(k * coord)
        U, T = rhs.init_state(mt, tensor(prim))
        out, _ = rhs.rhs(mt, GridT(n, n, 1, h, h, h), U, T, 0.0, None, fl)
        expect = factor * mu0 * eig * du * np.sin(k * coord) * np.ones((n, n))
        np.testing.assert_allclose(out[1, 0].numpy(), expect, rtol=1e-6, atol=1e-9 * abs(expect).max())


def _binary(W1, W2, D12=3e-5):
    a = np.zeros((2, 7))
    a[:, 0] = 3.5
    a[1, 5] = 2.0e4                       # different enthalpies: h_1 - h_2 enters the energy flux
    return synth.Mechanism(["A", "B"], np.array([W1, W2]), np.array([[1.0, 0], [0, 1.0]]), a.copy(), a.copy(),
                           np.full(2, 1000.0), np.full(2, 2e-5), np.full(2, 0.7),
                           np.array([[1e-5, D12], [D12, 1e-5]]), np.zeros(0), np.zeros(0), np.zeros(0),
                           np.zeros((0, 2), dtype=np.int64), np.zeros((0, 2), dtype=np.int64), np.zeros(0, dtype=np.int32))


def test_binary_diffusion_equal_molar_mass_closed_form():
    """Two species with equal W at uniform p and T: the mixture-averaged flux with
    correction velocity is Fick's law with D_12, so the species RHS is
    rho D_12 times the discrete Laplacian of Y_1, and the energy RHS is
    (h_1 - h_2) times the species RHS."""
    W = 0.02
    m = _binary(W, W)
    mt = mech_t(m)
    n, h = 32, 1e-4
    k = 2 * math.pi * 2 / (n * h)
    x = (np.arange(n) + 0.5) * h
    Y1 = 0.4 + 0.1 * np.sin(k * x)
    prim = np.zeros((7, 1, 1, n))
    prim[0], prim[1] = 101325.0, 500.0
    prim[5], prim[6] = Y1, 1.0 - Y1
    U, T = rhs.init_state(mt, tensor(prim))
    fl = {"inviscid": False, "chemistry": False, "laser": False}
    out, _ = rhs.rhs(mt, GridT(n, 1, 1, h, h, h), U, T, 0.0, None, fl)
    rho = 101325.0 * W / (R * 500.0)
    D12 = 3e-5 * (500.0 / 300.0) ** 1.75
    eig = -4.0 * math.sin(k * h / 2) ** 2 / h ** 2
    expect = rho * D12 * eig * 0.1 * np.sin(k * x)
    np.testing.assert_allclose(out[0, 0, 0].numpy(), expect, rtol=1e-9, atol=1e-10 * abs(expect).max())
    hs = thermo.species_h(mt, torch.tensor([500.0], dtype=torch.float64))[:, 0].numpy()
    np.testing.assert_allclose(out[5, 0, 0].numpy(), (hs[0] - hs[1]) * out[0, 0, 0].numpy(), rtol=1e-9,
                               atol=1e-9 * abs(hs[0] - hs[1]) * abs(expect).max())


def test_binary_diffusion_unequal_molar_mass_converges_to_fick():
    """W_1 != W_2: the species RHS converges at second order to the continuum
    d/dx(rho D_12 dY_1/dx) (binary Fick), which pins the W_s / Wbar factors."""
    W1, W2 = 0.004, 0.032
    m = _binary(W1, W2)
    mt = mech_t(m)
    L = 3.2e-3
    T0, p0 = 500.0, 101325.0
    D12 = 3e-5 * (T0 / 300.0) ** 1.75
    errs = []
    for n in (32, 64, 128):
        h = L / n
        x = (np.arange(n) + 0.5) * h
        k = 2 * math.pi / L
        Y1 = 0.5 + 0.3 * np.sin(k * x)
        dY = 0.3 * k * np.cos(k * x)
        d2Y = -0.3 * k * k * np.sin(k * x)
        Wb = 1.0 / (Y1 / W1 + (1 - Y1) / W2)
        rho = p0 * Wb / (R * T0)
        drho = rho * (-Wb) * (1 / W1 - 1 / W2) * dY     # d rho / dx at fixed p, T
        exact = D12 * (drho * dY + rho * d2Y)
        prim = np.zeros((7, 1, 1, n))
        prim[0], prim[1] = p0, T0
        prim[5], prim[6] = Y1, 1.0 - Y1
        U, T = rhs.init_state(mt, tensor(prim))
        out, _ = rhs.rhs(mt, GridT(n, 1, 1, h, h, h), U, T, 0.0, None,
                         {"inviscid": False, "chemistry": False, "laser": False})
        errs.append(np.abs(out[0, 0, 0].numpy() - exact).max() / np.abs(exact).max())
    assert errs[-1] < 1e-3
    for a, b in zip(errs[:-1], errs[1:]):
        assert math.log2(a / b) > 1.9


def test_sod_shock_tube_against_exact_riemann_solution():
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "sod_toro_test1.json")))
    g = gold["gamma"]
    L = (gold["left"]["rho"], gold["left"]["u"], gold["left"]["p"])
    Rt = (gold["right"]["rho"], gold["right"]["u"], gold["right"]["p"])
    ps, us = rx.star_state(L, Rt, g)
    assert abs(ps - gold["p_star"]) < 1e-5 and abs(us - gold["u_star"]) < 1e-5
    mt = mech_t(ca.gas())
    l1 = []
    for n in (200, 400):
        h = 1.0 / n
        x = (np.arange(n) + 0.5) * h
        left = x < 0.5
        rho0 = np.where(left, L[0], Rt[0])
        p0 = np.where(left, L[2], Rt[2])
        prim = np.zeros((6, 1, 1, n))
        prim[0] = p0
        prim[1] = p0 / rho0
        prim[5] = 1.0
        U, T = rhs.init_state(mt, tensor(prim))
        grid = GridT(n, 1, 1, h, h, h, (1, 0, 0))
        fl = {"viscous": False, "chemistry": False, "laser": False}
        t = 0.0
        while t < 0.2 - 1e-14:
            dt = min(rk.time_step(mt, grid, U, T, t, None, 0.5, fl), 0.2 - t)
            U, T, _ = rk.rk_step(mt, grid, U, T, t, dt, None, flags=fl)
            t += dt
        rho = U[0, 0, 0].numpy()
        u = U[1, 0, 0].numpy() / rho
        st = rhs.primitives(mt, U, T)
        p = st["p"][0, 0].numpy()
        ex = rx.sample(L, Rt, g, (x - 0.5) / t)
        l1.append(np.abs(rho - ex[0]).mean())
        if n == 400:
            xs = 0.5 + rx.shock_speed_right(L, Rt, g) * t
            band = (x > 0.5 + us * t + 0.03) & (x < xs - 0.02)
            assert abs(p[band].mean() - ps) < 0.01 * ps
            assert abs(u[band].mean() - us) < 0.01 * us
            mid = 0.5 * (ps + Rt[2])
            i = np.where((p[:-1] >= mid) & (p[1:] < mid) & (x[:-1] > 0.7))[0][0]
            xnum = x[i] + (p[i] - mid) / (p[i] - p[i + 1]) * h
            assert abs((xnum - 0.5) / t - rx.shock_speed_right(L, Rt, g)) < 0.01 * rx.shock_speed_right(L, Rt, g)
    assert l1[1] < 0.75 * l1[0]


def _vortex_errors(Ns, weights="weno"):
    mt = mech_t(ca.gas())
    errs = []
    orig = fluxes.weno3z
    if weights == "linear":          # WENO3-Z with its ideal weights d = (1/3, 2/3)
        fluxes.weno3z = lambda a, b, c, h: (1.0 / 3.0) * (-0.5 * a + 1.5 * b) + (2.0 / 3.0) * (0.5 * b + 0.5 * c)
    try:
        for N in Ns:
            prim, _, dx = ca.vortex_prim(N)
            g = GridT(N, N, 1, dx, dx, dx)
            U, T = rhs.init_state(mt, tensor(prim))
            t, dt = 0.0, 1e-3
            fl = {"viscous": False, "chemistry": False, "laser": False}
            for _ in range(50):
                U, T, _ = rk.rk_step(mt, g, U, T, t, dt, None, flags=fl)
                t += dt
            _, rex, _ = ca.vortex_prim(N, t)
            errs.append(np.abs(U[0, 0].numpy() - rex).mean())
    finally:
        fluxes.weno3z = orig
    return errs


def test_vortex_convergence_linear_weights_third_order():
    """Accuracy problem 1 (isentropic vortex, Cartesian, t = 0.05): with the ideal
    weights the split conservative scheme and RK3 converge at third order."""
    e = _vortex_errors((32, 64, 128), "linear")
    assert math.log2(e[1] / e[2]) > 2.6


def test_vortex_convergence_weno3z():
    """The same problem with the nonlinear WENO3-Z weights (p = 1, grid-scaled eps):
    third order, as the paper reports for WENO3-Z (Solver Performance Analysis,
    Accuracy), measured between N = 64 and N = 128 (2.95 with this eps; a fixed
    eps = 1e-30 gives 1.7 there, the weights losing accuracy at smooth extrema)."""
    e = _vortex_errors((32, 64, 128))
    assert math.log2(e[0] / e[1]) > 2.5 and math.log2(e[1] / e[2]) > 2.7
    assert e[2] < 2e-6


def test_taylor_green_second_order():
    """Accuracy problem 2 (2-D Taylor-Green, Re0 = L, Ma0 = 1e-2/sqrt(gamma),
    t = 0.05): the L1 error of u against the incompressible solution converges at
    least at second order (the paper's rate, set by the central viscous terms)
    from N = 16 to 32 (2.9 measured: at these resolutions the reconstruction error,
    third order, still dominates), and by N = 64 it reaches the O(Ma) floor of
    comparing a compressible run with the incompressible solution (1.5e-3 with
    either eps reading or the ideal weights)."""
    mt = mech_t(ca.gas(mu=1.0))
    errs = []
    for N in (16, 32, 64):
        prim, dx, _ = ca.tgv_prim(N)
        g = GridT(N, N, 1, dx, dx, dx)
        U, T = rhs.init_state(mt, tensor(prim))
        t = 0.0
        dt = rk.time_step(mt, g, U, T, 0.0, None, 0.5, NOSRC)
        nst = int(math.ceil(0.05 / dt))
        dt = 0.05 / nst
        for _ in range(nst):
            U, T, _ = rk.rk_step(mt, g, U, T, t, dt, None, flags=NOSRC)
            t += dt
        u = (U[1] / U[0])[0].numpy()
        errs.append(np.abs(u - ca.tgv_exact_u(N, t)).mean())
    assert math.log2(errs[0] / errs[1]) > 1.8
    assert errs[2] < 2e-3
