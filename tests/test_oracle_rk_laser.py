"""Pins of SSP-RK3, the laser source and the time-step rule."""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp

from paper_2202_02319_b300 import synth
from oracle import laser, rhs, rk, transport, thermo
from oracle.mech import GridT
from tests.helpers import mech_t, random_prim, tensor


@pytest.mark.parametrize("z", [-2.5, -1.0, -0.3, 0.1, 0.7])
def test_rk3_linear_amplification(z):
    """On dU/dt = lambda U one step multiplies by 1 + z + z^2/2 + z^3/6, z = lambda dt."""
    U = torch.tensor([1.0, -2.0], dtype=torch.float64)
    out = rk.ssp_rk3(lambda V, t: z * V, U, 0.0, 1.0)
    np.testing.assert_allclose(out.numpy(), U.numpy() * (1 + z + z * z / 2 + z ** 3 / 6), rtol=1e-15)


def test_rk3_third_order_in_time_with_stage_times():
    """A non-autonomous nonlinear scalar ODE converges at third order, which also
    pins the stage times t, t + dt, t + dt/2."""
    f = lambda y, t: -y * y + torch.sin(3.0 * t) if isinstance(y, torch.Tensor) else -y * y + math.sin(3.0 * t)
    ref = solve_ivp(lambda t, y: [-y[0] ** 2 + math.sin(3 * t)], (0, 1.0), [1.0], rtol=1e-13, atol=1e-14).y[0, -1]
    errs = []
    for n in (20, 40, 80):
        y = torch.tensor([1.0], dtype=torch.float64)
        t = 0.0
        for _ in range(n):
            y = rk.ssp_rk3(lambda v, tt: -v * v + math.sin(3.0 * tt), y, t, 1.0 / n)
            t += 1.0 / n
        errs.append(abs(float(y[0]) - ref))
    for a, b in zip(errs[:-1], errs[1:]):
        assert 2.8 < math.log2(a / b) < 3.3


@pytest.mark.parametrize("nz", [1, 48])
def test_laser_energy_integral(nz):
    """sum q_L dV = E_L exp(-(t-t0)^2 / 2 sigma_t^2) / (sqrt(2 pi) sigma_t) (per unit
    depth in 2-D), with the Gaussian well inside the box."""
    n, h = 48, 1e-4
    grid = GridT(n, n, nz, h, h, h)
    las = (0.02, 24.3 * h, 23.7 * h, 24.1 * h, 2.5 * h, 3e-8, 1e-8)
    for t in (3e-8, 4.1e-8, 1.5e-8):
        q = laser.laser_source(grid, t, las)
        vol = h * h * (h if nz > 1 else 1.0)
        expect = las[0] * math.exp(-0.5 * ((t - las[5]) / las[6]) ** 2) / (math.sqrt(2 * math.pi) * las[6])
        np.testing.assert_allclose(float(q.sum()) * vol, expect, rtol=1e-12)


def test_wilke_single_species_and_identical_species_split():
    """Wilke's rule returns mu_s for a pure species, and splitting one species into
    two identical copies does not change the mixture viscosity."""
    m = synth.mechanism_9sp(0)
    mt = mech_t(m)
    T = torch.tensor([300.0, 1200.0, 2500.0], dtype=torch.float64)
    mu_s = transport.species_viscosity(mt, T)
    phi = transport.wilke_phi(mt, mu_s)
    for s in range(9):
        X = torch.zeros(9, 3, dtype=torch.float64)
        X[s] = 1.0
        np.testing.assert_allclose(transport.wilke_mixture(X, mu_s, phi).numpy(), mu_s[s].numpy(), rtol=1e-15)
    # two identical copies of species 0
    W2 = np.array([m.W[0], m.W[0]])
    mu2 = torch.stack([mu_s[0], mu_s[0]])
    sub = mt.__class__(**{**mt.__dict__, "W": torch.tensor(W2)})
    phi2 = transport.wilke_phi(sub, mu2)
    X2 = torch.tensor([[0.3] * 3, [0.7] * 3], dtype=torch.float64)
    np.testing.assert_allclose(transport.wilke_mixture(X2, mu2, phi2).numpy(), mu_s[0].numpy(), rtol=1e-15)


def test_time_step_rule_components():
    """The rule returns the smallest of its limits, and the laser clamp holds dt to
    sigma_t/4 inside the pulse window and stops a step at the window's start."""
    c = synth.case_jet(0, 16)
    mt = mech_t(c.mech)
    from oracle.mech import grid_from_synth
    g = grid_from_synth(c.grid)
    U, T = rhs.init_state(mt, tensor(c.prim))
    ac, dmax, ch = rk.rate_limits(mt, g, U, T)
    base = min(0.5 / ac, 0.25 * g.dx ** 2 / dmax, 0.2 / ch if ch > 0 else 1e300)
    far = (0.01, 0, 0, 0, 1e-3, 1.0, 1e-8)
    assert rk.time_step(mt, g, U, T, 0.0, far, 0.5) == base
    inside = (0.01, 0, 0, 0, 1e-3, 1e-6, 1e-8)
    assert rk.time_step(mt, g, U, T, 1e-6 - 1e-8, inside, 0.5) == min(base, 0.25e-8)
    near = (0.01, 0, 0, 0, 1e-3, 6e-8 + 0.4 * base, 1e-8)
    assert rk.time_step(mt, g, U, T, 0.0, near, 0.5) == pytest.approx(0.4 * base, rel=1e-12)


def test_wilke_phi_reciprocity():
    """Wilke's interaction factors satisfy Phi_ji = Phi_ij mu_j W_i / (mu_i W_j), an
    identity that fixes the 1/2 and 1/4 exponents and the (1 + W_i/W_j) factor."""
    m = synth.mechanism_9sp(2)
    mt = mech_t(m)
    T = torch.tensor([350.0, 2200.0], dtype=torch.float64)
    mu = transport.species_viscosity(mt, T)
    phi = transport.wilke_phi(mt, mu)
    W = torch.tensor(m.W)
    for i in range(9):
        for j in range(9):
            np.testing.assert_allclose(phi[j, i].numpy(), (phi[i, j] * mu[j] * W[i] / (mu[i] * W[j])).numpy(), rtol=1e-14)
    np.testing.assert_allclose(torch.diagonal(phi).numpy(), 1.0, rtol=1e-15)
