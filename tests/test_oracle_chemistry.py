"""Pins of the oracle's chemistry: conservation laws, a closed-form relaxation,
the Jacobian diagonal used by the time-step rule, and a homogeneous reactor
against a stiff brute-force integration."""
import math

import numpy as np
import pytest
import torch
from scipy.integrate import solve_ivp

from paper_2202_02319_b300 import synth
from oracle import chemistry, rhs, rk, thermo
from oracle.mech import GridT
from tests.helpers import mech_t, tensor, R



def _random_state(m, n, seed):
    g = np.random.default_rng(seed)
    rho_s = g.uniform(0.0, 1.0, (m.n_species, n)) * g.uniform(0.05, 3.0, n)
    T = g.uniform(600.0, 3500.0, n)
    return tensor(rho_s), tensor(T)


@pytest.mark.parametrize("mk", [synth.mechanism_4sp, synth.mechanism_9sp, synth.mechanism_9sp_pressure])
def test_mass_and_element_conservation(mk):
    m = mk(0)
    mt = mech_t(m)
    rho_s, T = _random_state(m, 500, 4)
    w = chemistry.production_rates(mt, rho_s, T)
    scale = w.abs().sum(0) + 1e-300
    assert float((w.sum(0).abs() / scale).max()) < 1e-13
    el = tensor(m.elem).T @ (w / tensor(m.W)[:, None])                    # mol of element / m^3 / s
    elscale = (tensor(m.elem).T @ (w.abs() / tensor(m.W)[:, None])) + 1e-300
    assert float((el.abs() / elscale).max()) < 1e-13


def _two_species_isomer(kf_A, b, Theta, s_A, s_B, W=0.03):
    """A <=> B with identical W, cp and formation enthalpy: no heat release, so T
    stays fixed, and K_c = exp((s_B - s_A) / R)."""
    a = np.zeros((2, 7))
    a[:, 0] = 3.5
    a[:, 6] = np.array([s_A, s_B]) / R - 3.5 * np.log(298.15)
    return synth.Mechanism(["A", "B"], np.array([W, W]), np.array([[1.0], [1.0]]), a.copy(), a.copy(),
                           np.full(2, 1000.0), np.full(2, 2e-5), np.full(2, 0.7), np.full((2, 2), 2e-5),
                           np.array([kf_A]), np.array([b]), np.array([Theta]),
                           np.array([[1, 0]]), np.array([[0, 1]]), np.array([1], dtype=np.int32))


def test_isomerisation_relaxes_with_closed_form():
    """Homogeneous A <=> B at fixed T: C_A(t) = C_eq + (C_A0 - C_eq) exp(-(k_f + k_r) t)
    with k_r = k_f exp(-(s_B - s_A)/R); integrated by the oracle's own RK3 step on a
    one-cell periodic box, it must equal the RK3 amplification factor
    (1 + z + z^2/2 + z^3/6)^n of that linear ODE to rounding."""
    T0 = 1200.0
    A, b, Th = 5.0e4, 0.5, 8000.0
    sA, sB = 180.0, 190.0
    m = _two_species_isomer(A, b, Th, sA, sB)
    mt = mech_t(m)
    grid = GridT(1, 1, 1, 1e-3, 1e-3, 1e-3)
    prim = np.array([101325.0, T0, 0.0, 0.0, 0.0, 1.0, 0.0]).reshape(7, 1, 1, 1)
    U, T = rhs.init_state(mt, tensor(prim))
    kf = A * T0 ** b * math.exp(-Th / T0)
    kr = kf * math.exp(-(sB - sA) / R)
    rho = float(U[:2].sum())
    CA0 = rho / 0.03
    Ceq = CA0 * kr / (kf + kr)
    dt = 0.02 / (kf + kr)
    t = 0.0
    for _ in range(150):
        U, T, _ = rk.rk_step(mt, grid, U, T, t, dt, None, flags={"laser": False})
        t += dt
    CA = float(U[0]) / 0.03
    z = -(kf + kr) * dt
    discrete = Ceq + (CA0 - Ceq) * (1.0 + z + z * z / 2.0 + z ** 3 / 6.0) ** 150
    exact = Ceq + (CA0 - Ceq) * math.exp(-(kf + kr) * t)
    assert abs(CA - discrete) / CA0 < 1e-12          # RK3 on a linear ODE, to rounding
    assert abs(CA - exact) / CA0 < 1e-7              # and the continuous solution, to O(dt^3)
    assert abs(float(T.flatten()[0]) - T0) < 1e-9 * T0


@pytest.mark.parametrize("mk", [synth.mechanism_4sp, synth.mechanism_9sp])
def test_chemical_rate_is_jacobian_diagonal(mk):
    """max_s |d omega_s / d rho_s| matches central differences of omega at fixed T."""
    m = mk(1)
    mt = mech_t(m)
    rho_s, T = _random_state(m, 50, 5)
    est = chemistry.chemical_rate(mt, rho_s, T)
    fd = torch.zeros_like(T)
    for s in range(m.n_species):
        h = 1e-6 * (rho_s[s] + 1e-3)
        rp = rho_s.clone(); rp[s] += h
        rm = rho_s.clone(); rm[s] -= h
        d = (chemistry.production_rates(mt, rp, T)[s] - chemistry.production_rates(mt, rm, T)[s]) / (2 * h)
        fd = torch.maximum(fd, d.abs())
    np.testing.assert_allclose(est.numpy(), fd.numpy(), rtol=1e-5)


@pytest.mark.parametrize("mk", [synth.mechanism_9sp, synth.mechanism_9sp_pressure])
def test_homogeneous_reactor_against_stiff_integration(mk):
    """A uniform 4^3 periodic box evolves as a constant-volume reactor: the RK3
    trajectory at a chemically resolved dt matches a Radau integration of
    d rho_s/dt = omega_s(rho, e) to 1e-6, total energy is constant and the box stays
    uniform (elementary reactions, and with third-body and fall-off reactions)."""
    m = mk(0)
    mt = mech_t(m)
    n = 4
    grid = GridT(n, n, n, 1e-4, 1e-4, 1e-4)
    Y = np.zeros(9)
    Y[m.index("X2")] = 0.05
    Y[m.index("Y2")] = 0.2
    Y[m.index("Z2")] = 0.7
    Y[m.index("X")] = 0.02
    Y[m.index("XY")] = 0.03
    Y /= Y.sum()
    prim = np.concatenate([[101325.0, 1500.0, 0.0, 0.0, 0.0], Y]).reshape(-1, 1, 1, 1) * np.ones((1, n, n, n))
    U, T = rhs.init_state(mt, tensor(prim))
    E0 = float(U[-1].sum())
    rho = float(U[:9, 0, 0, 0].sum())
    e_int = float(U[-1, 0, 0, 0]) / rho

    def f(_, y):
        rs = tensor(y[:, None])
        Yc = rs / rs.sum(0)
        Tc, _, _ = thermo.temperature_from_energy(mt, Yc, torch.tensor([e_int], dtype=torch.float64),
                                                  torch.tensor([1500.0], dtype=torch.float64))
        return chemistry.production_rates(mt, rs, Tc)[:, 0].numpy()
    rate0 = float(chemistry.chemical_rate(mt, U[:9, 0:1, 0:1, 0:1].reshape(9, 1), T[0:1, 0, 0].reshape(1)))
    dt = 0.2 / rate0
    nsteps = 100
    t = 0.0
    flags = {"laser": False}
    for _ in range(nsteps):
        U, T, _ = rk.rk_step(mt, grid, U, T, t, dt, None, flags=flags)
        t += dt
    sol = solve_ivp(f, (0.0, t), U[:9, 0, 0, 0].numpy() * 0 + prim[5:, 0, 0, 0] * rho, method="Radau",
                    rtol=1e-12, atol=1e-14 * rho)
    ref = sol.y[:, -1]
    got = U[:9, 0, 0, 0].numpy()
    assert np.max(np.abs(got - ref)) / rho < 1e-6
    assert abs(float(U[-1].sum()) - E0) <= 1e-13 * abs(E0)
    assert float((U - U[:, :1, :1, :1]).abs().max()) == 0.0
    assert abs(float(T[0, 0, 0]) - 1500.0) > 0.1            # the reactor really reacted
