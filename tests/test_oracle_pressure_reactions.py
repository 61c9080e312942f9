"""Pins of the oracle's pressure-dependent reactions (third body, Lindemann and
Troe fall-off; the paper's CH4/O2 mechanisms, Methods - Combustion chemistry,
use them without printing them): the third-body concentration of unit
efficiencies is the ideal-gas total p / (R T), the fall-off rate meets its two
pressure limits, the Troe factor equals F_c at the centre of its broadening
curve and tends to one away from it, and equilibrium compositions give zero net
rate for every reaction type."""
import math

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import chemistry, thermo
from tests.helpers import mech_t, tensor, R


def _dimer(kind, eff=(1.0, 1.0), A0=3.0e4, b0=-0.7, Th0=2500.0, troe=(0.6, 200.0, 1500.0, 4000.0)):
    """2A <=> B (W_B = 2 W_A) with one reaction of the given kind."""
    W = np.array([0.016, 0.032])
    cp = np.array([3.5, 4.5])
    a = np.zeros((2, 7))
    a[:, 0] = cp
    a[:, 5] = np.array([0.0, -150e3]) / R - cp * 298.15
    a[:, 6] = np.array([160.0, 230.0]) / R - cp * math.log(298.15)
    m = synth.Mechanism(["A", "B"], W, np.array([[1.0], [2.0]]), a.copy(), a.copy(), np.full(2, 1000.0),
                        np.full(2, 2e-5), np.full(2, 0.7), np.full((2, 2), 2e-5),
                        np.array([2.0e6]), np.array([0.3]), np.array([6000.0]),
                        np.array([[2, 0]]), np.array([[0, 1]]), np.array([1], dtype=np.int32))
    if kind:
        m.rxn_type = np.array([kind], dtype=np.int32)
        m.efficiency = np.array([eff], dtype=float)
        m.A0, m.b0, m.Theta0 = np.array([A0]), np.array([b0]), np.array([Th0])
        m.troe = np.array([troe], dtype=float)
    return m


def _state(n=6, seed=0):
    g = np.random.default_rng(seed)
    C = tensor(g.uniform(0.5, 20.0, (2, n)))
    T = tensor(g.uniform(600.0, 2500.0, n))
    return C, T


def test_third_body_with_unit_efficiencies_is_the_total_concentration():
    """With every efficiency 1, [M] = sum C_s = rho / Wbar = p / (R T): the rate of
    progress is the elementary one times the total molar concentration from the
    equation of state."""
    C, T = _state()
    q0, _, _ = chemistry.rates_of_progress(mech_t(_dimer(0)), C, T)
    q1, _, _ = chemistry.rates_of_progress(mech_t(_dimer(1)), C, T)
    W = tensor(np.array([0.016, 0.032]))
    rho_s = C * W[:, None]
    rho = rho_s.sum(0)
    p = thermo.pressure(mech_t(_dimer(0)), rho, rho_s / rho, T)
    assert float(((q1 / q0) / (p / (R * T)) - 1.0).abs().max()) < 1e-13


def test_third_body_efficiencies_weight_the_species():
    """Efficiencies (2.5, 0.4): the factor is 2.5 C_A + 0.4 C_B."""
    C, T = _state(seed=1)
    q0, _, _ = chemistry.rates_of_progress(mech_t(_dimer(0)), C, T)
    q1, _, _ = chemistry.rates_of_progress(mech_t(_dimer(1, eff=(2.5, 0.4))), C, T)
    assert float(((q1 / q0) / (2.5 * C[0] + 0.4 * C[1]) - 1.0).abs().max()) < 1e-13


@pytest.mark.parametrize("kind", [2, 3])
def test_fall_off_meets_both_pressure_limits(kind):
    """The fall-off rate constant over its broadening factor tends to k_inf at high
    [M] and to k_0 [M] at low [M] (to the order of 1 / P_r or P_r), for Lindemann
    (F = 1) and Troe."""
    m = mech_t(_dimer(kind))
    T = tensor(np.array([800.0, 1500.0, 2200.0]))
    kinf = 2.0e6 * T ** 0.3 * torch.exp(-6000.0 / T)
    k0 = 3.0e4 * T ** -0.7 * torch.exp(-2500.0 / T)
    for scale, expect in ((1e9, lambda M: kinf), (1e-9, lambda M: k0 * M)):
        C = torch.stack([torch.full_like(T, 3.0), torch.full_like(T, 1.0)]) * scale
        M = C.sum(0)
        _, fwd, _ = chemistry.rates_of_progress(m, C, T)
        Pr = k0 * M / kinf
        F = chemistry.troe_factor(m, 0, T, Pr) if kind == 3 else 1.0
        k = fwd[0] / (C[0] * C[0]) / F
        tol = 1e-5 + 5.0 * float(torch.minimum(Pr, 1.0 / Pr).max())
        assert float((k / expect(M) - 1.0).abs().max()) < tol


def test_troe_factor_centre_and_wings():
    """F = F_c where log10 P_r = -c (the centre of the broadening curve); far from it
    on both sides log10 P_r + c over n - 0.14 (log10 P_r + c) tends to -1/0.14, so F
    tends to F_c^(1 / (1 + 1/0.14^2))."""
    m = mech_t(_dimer(3))
    T = tensor(np.array([700.0, 1300.0, 2100.0]))
    al, T3, T1, T2 = 0.6, 200.0, 1500.0, 4000.0
    Fc = (1 - al) * torch.exp(-T / T3) + al * torch.exp(-T / T1) + torch.exp(-T2 / T)
    c = -0.4 - 0.67 * torch.log10(Fc)
    F = chemistry.troe_factor(m, 0, T, 10.0 ** (-c))
    assert float((F / Fc - 1.0).abs().max()) < 1e-13
    wing = Fc ** (1.0 / (1.0 + 1.0 / 0.14 ** 2))
    for sgn in (-1.0, 1.0):
        far = chemistry.troe_factor(m, 0, T, torch.full_like(T, 10.0 ** (sgn * 250.0)))
        near = chemistry.troe_factor(m, 0, T, torch.full_like(T, 10.0 ** (sgn * 25.0)))
        assert float((far / wing - 1.0).abs().max()) < 3e-3
        assert bool(((far - wing).abs() < (near - wing).abs()).all())
    assert bool((F < 1.0).all())


@pytest.mark.parametrize("kind", [1, 2, 3])
def test_equilibrium_composition_has_zero_net_rate(kind):
    """C_B = K_c C_A^2 from the equilibrium constant gives q = 0 to rounding for
    every reaction type (the pressure dependence multiplies both directions)."""
    m = mech_t(_dimer(kind, eff=(1.7, 0.6)))
    T = tensor(np.array([900.0, 1400.0, 2300.0]))
    Kc = chemistry.equilibrium_constants(m, T)[0]
    CA = tensor(np.array([2.0, 0.5, 7.0]))
    C = torch.stack([CA, Kc * CA * CA])
    q, fwd, _ = chemistry.rates_of_progress(m, C, T)
    assert float((q[0].abs() / fwd[0].abs()).max()) < 1e-13
