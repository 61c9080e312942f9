"""Pins of the oracle's thermodynamics (NASA-7 forms, EOS, temperature Newton)
against closed forms and calculus, not against the oracle itself."""
import numpy as np
import pytest
import torch
from scipy import integrate

from paper_2202_02319_b300 import synth
from oracle import thermo, chemistry, rhs
from tests.helpers import mech_t, tensor, R



def test_constant_cp_closed_form_temperature():
    """Constant cp: e(T) is linear, so T = (e - sum Y e0_s) / cv exactly and Newton
    lands there in one update (the second only confirms convergence)."""
    m = synth.mechanism_4sp(0)
    mt = mech_t(m)
    g = np.random.default_rng(1)
    Y = g.dirichlet(np.ones(4), size=64).T
    T_true = g.uniform(250.0, 3000.0, 64)
    cv = (m.nasa_low[:, 0] - 1.0) * R / m.W                  # J/kg/K
    e0 = m.nasa_low[:, 5] * R / m.W                           # e_s = cv_s T + R a6 / W_s
    e = (Y * (cv[:, None] * T_true + e0[:, None])).sum(0)
    T, conv, its = thermo.temperature_from_energy(mt, tensor(Y), tensor(e), torch.full((64,), 1000.0))
    assert bool(conv.all())
    assert int(its.max()) <= 2
    np.testing.assert_allclose(T.numpy(), (e - (Y * e0[:, None]).sum(0)) / (Y * cv[:, None]).sum(0), rtol=1e-13)
    np.testing.assert_allclose(T.numpy(), T_true, rtol=1e-12)


def test_newton_round_trip_nasa7():
    """T -> e(T) -> Newton from a distant guess returns T to 1e-13."""
    m = synth.mechanism_9sp(0)
    mt = mech_t(m)
    g = np.random.default_rng(2)
    Y = g.dirichlet(np.ones(9), size=200).T
    T_true = g.uniform(220.0, 5000.0, 200)
    e = (tensor(Y) * thermo.species_e(mt, tensor(T_true))).sum(0)
    T, conv, _ = thermo.temperature_from_energy(mt, tensor(Y), e, torch.full((200,), 1500.0))
    assert bool(conv.all())
    np.testing.assert_allclose(T.numpy(), T_true, rtol=1e-13)


def test_enthalpy_and_entropy_are_integrals_of_cp():
    """dh/dT = cp and ds/dT = cp/T (finite differences of the oracle's h and s),
    and h, s at 298.15 K equal the integrals of cp added to the reference values."""
    m = synth.mechanism_9sp(3)
    mt = mech_t(m)
    T = torch.linspace(300.0, 5000.0, 40, dtype=torch.float64)
    d = 1e-3
    dh = (thermo.species_h(mt, T + d) - thermo.species_h(mt, T - d)) / (2 * d)
    np.testing.assert_allclose(dh.numpy(), thermo.species_cp(mt, T).numpy(), rtol=1e-7)
    ds = (thermo.s_R(mt, T + d) - thermo.s_R(mt, T - d)) / (2 * d)
    np.testing.assert_allclose(ds.numpy(), (thermo.cp_R(mt, T) / T).numpy(), rtol=1e-7)
    for s in range(9):
        cpR = lambda x: float(thermo.cp_R(mt, torch.tensor([x], dtype=torch.float64))[s, 0])
        Ia, _ = integrate.quad(cpR, 298.15, 2000.0, epsabs=0, epsrel=1e-13)
        hT = thermo.h_RT(mt, torch.tensor([298.15, 2000.0], dtype=torch.float64))[s]
        np.testing.assert_allclose(float(hT[1]) * 2000.0 - float(hT[0]) * 298.15, Ia, rtol=1e-11)


def test_equilibrium_constant_from_gibbs_energy_by_quadrature():
    """K_c from Delta G = Delta H - T Delta S with H and S integrated from cp by
    quadrature starting at the 298.15 K values; an equilibrium composition built
    from it gives zero net rate of progress."""
    m = synth.mechanism_9sp(0)
    mt = mech_t(m)
    Tref = 298.15
    Tq = 1700.0
    tr = torch.tensor([Tref], dtype=torch.float64)
    H, S = [], []
    for s in range(9):
        cpR = lambda x: float(thermo.cp_R(mt, torch.tensor([x], dtype=torch.float64))[s, 0])
        h0 = float(thermo.h_RT(mt, tr)[s, 0]) * R * Tref
        s0 = float(thermo.s_R(mt, tr)[s, 0]) * R
        H.append(h0 + R * integrate.quad(cpR, Tref, Tq, epsrel=1e-13)[0])
        S.append(s0 + R * integrate.quad(lambda x: cpR(x) / x, Tref, Tq, epsrel=1e-13)[0])
    H, S = np.array(H), np.array(S)
    dnu = m.nu_r - m.nu_f
    dG = dnu @ (H - Tq * S)
    Kc_ref = np.exp(-dG / (R * Tq)) * (101325.0 / (R * Tq)) ** dnu.sum(1)
    Kc = chemistry.equilibrium_constants(mt, torch.tensor([Tq], dtype=torch.float64))[:, 0].numpy()
    np.testing.assert_allclose(Kc, Kc_ref, rtol=1e-9)
    # equilibrium composition for each reaction: scale the products to satisfy K_c
    for j in range(m.n_reactions):
        C = np.full(9, 2.0)
        n_prod = m.nu_r[j].sum()
        prod_rest = np.prod([C[s] ** m.nu_f[j, s] for s in range(9)]) * Kc_ref[j]
        x = prod_rest ** (1.0 / n_prod)             # all products at the same concentration x
        for s in range(9):
            if m.nu_r[j, s]:
                C[s] = x
        q, f, r = chemistry.rates_of_progress(mt, tensor(C[:, None]), torch.tensor([Tq], dtype=torch.float64))
        assert abs(float(q[j, 0])) <= 1e-9 * float(f[j, 0])


def test_eos_and_sound_speed_single_gas():
    """p = rho R T / W and c = sqrt(gamma R T / W) for a calorically perfect gas."""
    from tests.helpers import single_species
    m = single_species(gamma=1.4, W=0.029)
    mt = mech_t(m)
    prim = np.array([[[[2.0e5]]], [[[600.0]]], [[[10.0]]], [[[0.0]]], [[[0.0]]], [[[1.0]]]])
    U, T = rhs.init_state(mt, tensor(prim))
    st = rhs.primitives(mt, U, T)
    rho = 2.0e5 * 0.029 / (R * 600.0)
    np.testing.assert_allclose(float(st["rho"]), rho, rtol=1e-15)
    np.testing.assert_allclose(float(st["p"]), 2.0e5, rtol=1e-13)
    np.testing.assert_allclose(float(st["c"]), np.sqrt(1.4 * R * 600.0 / 0.029), rtol=1e-13)
    np.testing.assert_allclose(float(U[4]), rho * (600.0 * R / 0.029 / 0.4 + 50.0), rtol=1e-13)
