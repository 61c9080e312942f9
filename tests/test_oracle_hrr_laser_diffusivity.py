"""Pins of three oracle functions against results fixed outside the oracle:

  * heat_release_rate (Methods, Combustion chemistry; the sensitivity objective of
    Application examples): the closed-form molar enthalpies of a constant-cp
    dimerisation 2A <=> B, and the energy equation of a constant-volume reactor;
  * laser_source (Methods, Diffusion flame, Eq. laser-qs): first and second
    moments of the deposited power, which fix the pulse centre (cell centres at
    (i + 1/2) h, axes not swapped) and its width;
  * mixture_diffusivity (Methods, Governing equations): Blanc's law for a trace
    species, equal molar masses with equal binary diffusivities, and the binary
    reduction, with three and four species and unequal coefficients.
"""
import math

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import chemistry, laser, thermo, transport
from oracle.mech import GridT
from tests.helpers import mech_t, tensor, R

T_REF = 298.15


def _dimerisation(cpA=3.5, cpB=4.5, HfA=0.0, HfB=-150.0e3, A=2.0e6, b=0.3, Theta=6000.0):
    """2A <=> B with W_B = 2 W_A and constant cp: molar enthalpy
    H_s(T) = H_f,s + R cp_s/R (T - 298.15), so a6 = H_f/R - a1 298.15."""
    W = np.array([0.016, 0.032])
    cp = np.array([cpA, cpB])
    Hf = np.array([HfA, HfB])
    s0 = np.array([160.0, 230.0])
    a = np.zeros((2, 7))
    a[:, 0] = cp
    a[:, 5] = Hf / R - cp * T_REF
    a[:, 6] = s0 / R - cp * math.log(T_REF)
    m = synth.Mechanism(["A", "B"], W, np.array([[1.0], [2.0]]), a.copy(), a.copy(),
                        np.full(2, 1000.0), np.full(2, 2e-5), np.full(2, 0.7), np.full((2, 2), 2e-5),
                        np.array([A]), np.array([b]), np.array([Theta]),
                        np.array([[2, 0]]), np.array([[0, 1]]), np.array([1], dtype=np.int32))
    return m, W, cp, Hf


def test_heat_release_rate_of_a_dimerisation_closed_form():
    """HRR = -sum_s h_s omega_s with omega_A = -2 W_A q, omega_B = W_B q is
    q (2 H_A(T) - H_B(T)) in molar enthalpies: positive for the exothermic
    forward direction, and it changes sign with q."""
    m, W, cp, Hf = _dimerisation()
    mt = mech_t(m)
    T = tensor(np.array([300.0, 650.0, 1200.0, 2400.0, 3300.0]))
    q = tensor(np.array([3.7, -0.25, 1.0e3, 42.0, -7.5e-2]))
    omega = torch.stack([-2.0 * W[0] * q, W[1] * q])
    H = [Hf[s] + R * cp[s] * (T - T_REF) for s in range(2)]
    expected = q * (2.0 * H[0] - H[1])
    got = chemistry.heat_release_rate(mt, omega, T)
    assert float(((got - expected).abs() / expected.abs()).max()) < 1e-13
    assert bool(((got > 0) == (q > 0)).all())


def test_heat_release_rate_drives_the_constant_volume_energy_balance():
    """In a closed constant-volume cell E is fixed, so rho c_v dT/dt =
    -sum_s e_s omega_s = HRR + R T sum_s omega_s / W_s (e_s = h_s - R T / W_s).
    dT/dt by central differences of the Newton temperature along omega must
    match that right-hand side; forward reaction exothermic, so T rises."""
    m, W, cp, Hf = _dimerisation()
    mt = mech_t(m)
    rho_s = tensor(np.array([[0.20, 0.05, 0.31], [0.02, 0.10, 0.01]]))
    T0 = tensor(np.array([1500.0, 1100.0, 2000.0]))
    omega = chemistry.production_rates(mt, rho_s, T0)
    rho = rho_s.sum(0)
    e = (rho_s * thermo.species_e(mt, T0)).sum(0) / rho
    hrr = chemistry.heat_release_rate(mt, omega, T0)
    rhs = hrr + R * T0 * (omega / tensor(W)[:, None]).sum(0)
    cv = (rho_s / rho * R * (tensor(cp)[:, None] - 1.0) / tensor(W)[:, None]).sum(0)
    dTdt_expected = rhs / (rho * cv)
    delta = 1e-6 * float((rho_s / omega.abs()).min())
    Tp, okp, _ = thermo.temperature_from_energy(mt, (rho_s + delta * omega) / rho, e, T0)
    Tm, okm, _ = thermo.temperature_from_energy(mt, (rho_s - delta * omega) / rho, e, T0)
    assert bool(okp.all()) and bool(okm.all())
    dTdt = (Tp - Tm) / (2.0 * delta)
    assert float(((dTdt - dTdt_expected).abs() / dTdt_expected.abs()).max()) < 1e-6
    q = -omega[0] / (2.0 * W[0])
    assert bool(((hrr > 0) == (q > 0)).all())
    assert bool((dTdt[q > 0] > 0).all())


def _moments(grid, las, t):
    q = laser.laser_source(grid, t, las)
    X, Y, Z = laser.cell_centres(grid)
    w = q / q.sum()
    return q, [float((w * C).sum()) for C in (X, Y, Z)], [float((w * C * C).sum()) for C in (X, Y, Z)]


def test_laser_first_and_second_moments_3d():
    """Off-centre pulse on an anisotropic grid: the power-weighted mean position is
    (x0, y0, z0) and the variance along each axis sigma_r^2 (the sampled Gaussian's
    moments equal the continuous ones to exp(-2 pi^2 sigma^2 / h^2), the pulse sits
    8 sigma inside the box)."""
    g = GridT(64, 56, 48, 1.0e-4, 1.2e-4, 0.9e-4)
    sr = 2.5e-4
    x0, y0, z0 = 30.3e-4, 27.6 * 1.2e-4, 23.4 * 0.9e-4
    las = (3.0e-3, x0, y0, z0, sr, 5e-8, 1e-8)
    q, m1, m2 = _moments(g, las, 5.3e-8)
    for c, mu, L in zip(m1, (x0, y0, z0), (64e-4, 56 * 1.2e-4, 48 * 0.9e-4)):
        assert abs(c - mu) < 1e-12 * L
    for c2, c1 in zip(m2, m1):
        assert abs((c2 - c1 * c1) / sr ** 2 - 1.0) < 1e-9
    dV = g.dx * g.dy * g.dz
    expect = las[0] * math.exp(-0.5 * ((5.3e-8 - 5e-8) / 1e-8) ** 2) / (math.sqrt(2 * math.pi) * 1e-8)
    assert abs(float(q.sum()) * dV / expect - 1.0) < 1e-12


def test_laser_first_and_second_moments_2d():
    """nz = 1: the paper's two-dimensional form, r in the x-y plane, z0 ignored."""
    g = GridT(72, 60, 1, 1.1e-4, 0.8e-4, 1e-4)
    sr = 3.0e-4
    x0, y0 = 40.7 * 1.1e-4, 29.6 * 0.8e-4
    las = (1.5e-3, x0, y0, 123.0, sr, 0.0, 1e-8)
    q, m1, m2 = _moments(g, las, 0.0)
    assert abs(m1[0] - x0) < 1e-12 * 72 * 1.1e-4
    assert abs(m1[1] - y0) < 1e-12 * 60 * 0.8e-4
    for c2, c1 in zip(m2[:2], m1[:2]):
        assert abs((c2 - c1 * c1) / sr ** 2 - 1.0) < 1e-9
    expect = las[0] / (math.sqrt(2 * math.pi) * 1e-8)
    assert abs(float(q.sum()) * g.dx * g.dy / expect - 1.0) < 1e-12


def _mech_D(W, Dref):
    ns = len(W)
    W = np.asarray(W, dtype=float)
    a = np.zeros((ns, 7))
    a[:, 0] = 3.5
    return synth.Mechanism([f"S{i}" for i in range(ns)], W, np.eye(ns), a.copy(), a.copy(),
                           np.full(ns, 1000.0), np.full(ns, 2e-5), np.full(ns, 0.7), np.asarray(Dref, dtype=float),
                           np.zeros(0), np.zeros(0), np.zeros(0), np.zeros((0, ns), dtype=np.int64),
                           np.zeros((0, ns), dtype=np.int64), np.zeros(0, dtype=np.int32))


def _sym(rng, ns, lo=1e-5, hi=8e-5):
    D = rng.uniform(lo, hi, (ns, ns))
    return np.triu(D) + np.triu(D, 1).T


@pytest.mark.parametrize("ns", [3, 4])
def test_mixture_diffusivity_trace_species_follows_blancs_law(ns):
    """A species absent from the mixture (X_s = 0) diffuses with Blanc's law
    1 / D_s = sum_{j != s} X_j / D_sj, whatever the molar masses."""
    rng = np.random.default_rng(ns)
    W = rng.uniform(0.002, 0.044, ns)
    D = _sym(rng, ns)
    mt = mech_t(_mech_D(W, D))
    for s in range(ns):
        X = rng.dirichlet(np.ones(ns - 1), size=5).T
        X = np.insert(X, s, 0.0, axis=0)
        Dij = tensor(D)[:, :, None]
        got = transport.mixture_diffusivity(mt, tensor(X), Dij.expand(ns, ns, 5))[s]
        blanc = 1.0 / sum(X[j] / D[s, j] for j in range(ns) if j != s)
        assert float((got - tensor(blanc)).abs().max() / blanc.max()) < 1e-10


def test_mixture_diffusivity_equal_molar_masses_and_equal_binaries():
    """Equal molar masses (Y = X) and one binary diffusivity D for every pair:
    every species diffuses with D."""
    rng = np.random.default_rng(7)
    ns = 4
    W = np.full(ns, 0.028)
    D = np.full((ns, ns), 3.3e-5)
    mt = mech_t(_mech_D(W, D))
    X = rng.dirichlet(np.ones(ns), size=9).T
    got = transport.mixture_diffusivity(mt, tensor(X), tensor(D)[:, :, None].expand(ns, ns, 9))
    assert float((got / 3.3e-5 - 1.0).abs().max()) < 1e-10


def test_mixture_diffusivity_reduces_to_the_binary_value():
    """Three species with the third absent: the two present ones diffuse with
    (1 - Y_1) / (X_2 / D_12) = D_12 W_2 / Wbar, the third with Blanc's law."""
    W = np.array([0.004, 0.032, 0.018])
    D = np.array([[1e-5, 6.1e-5, 2.2e-5], [6.1e-5, 1e-5, 4.4e-5], [2.2e-5, 4.4e-5, 1e-5]])
    mt = mech_t(_mech_D(W, D))
    x1 = np.array([0.1, 0.45, 0.8])
    X = np.stack([x1, 1.0 - x1, np.zeros(3)])
    got = transport.mixture_diffusivity(mt, tensor(X), tensor(D)[:, :, None].expand(3, 3, 3))
    Wbar = x1 * W[0] + (1.0 - x1) * W[1]
    assert float((got[0] / tensor(D[0, 1] * W[1] / Wbar) - 1.0).abs().max()) < 1e-10
    assert float((got[1] / tensor(D[0, 1] * W[0] / Wbar) - 1.0).abs().max()) < 1e-10
    blanc = 1.0 / (x1 / D[2, 0] + (1.0 - x1) / D[2, 1])
    assert float((got[2] / tensor(blanc) - 1.0).abs().max()) < 1e-10
