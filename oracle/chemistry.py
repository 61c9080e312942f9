"""Finite-rate reversible Arrhenius chemistry (Methods, Combustion chemistry).

The paper models the chemical source omega_s with finite-rate Arrhenius
reactions and omits the mechanism details.  Reading (standard mass-action
kinetics, no third-body or fall-off terms):

  C_s     = rho_s / W_s                                   [mol/m^3]
  k_f,j   = A_j T^b_j exp(-Theta_j / T)
  K_c,j   = exp(-sum_s nu_sj g_s/RT) (p_atm / (R T))^(sum_s nu_sj),
            nu_sj = nu''_sj - nu'_sj,  g_s/RT = h_s/RT - s_s/R (NASA polynomials)
  k_r,j   = k_f,j / K_c,j   (0 for an irreversible reaction)
  q_j     = k_f,j prod_s C_s^nu'_sj - k_r,j prod_s C_s^nu''_sj
  omega_s = W_s sum_j nu_sj q_j                           [kg/m^3/s]
  HRR     = -sum_s h_s omega_s                            [W/m^3]

Concentration products are formed by repeated multiplication over the
species that take part, so that species with zero coefficient never enter.

Pressure-dependent reactions (the paper's CH4/O2 mechanisms use them and omits
the details; reading: the CHEMKIN conventions):
  third body:  q_j = [M]_j (k_f prod C^nu' - k_r prod C^nu''),  [M]_j = sum_s eps_sj C_s
  fall-off:    k_f = k_inf P_r / (1 + P_r) F,  P_r = k_0 [M]_j / k_inf, with
               k_inf = A T^b exp(-Theta/T), k_0 = A0 T^b0 exp(-Theta0/T);
               Lindemann F = 1; Troe
               log10 F = log10 F_c / (1 + ((log10 P_r + c) / (n - 0.14 (log10 P_r + c)))^2),
               F_c = (1 - alpha) exp(-T/T***) + alpha exp(-T/T*) + exp(-T**/T),
               c = -0.4 - 0.67 log10 F_c, n = 0.75 - 1.27 log10 F_c;
               no further [M] factor; k_r = k_f / K_c as for every reaction.
The chemical time-step estimate (chemical_rate) differentiates at fixed [M]_j
and fixed fall-off factor.
"""
from __future__ import annotations

import torch

from .mech import P_ATM, R_U, MechT
from .thermo import _bcast, h_RT, s_R, species_h


def forward_rate_constants(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """k_f [Nr, ...] of the Arrhenius form (for a fall-off reaction, its
    high-pressure limit k_inf)."""
    A = _bcast(mech.A, T)
    b = _bcast(mech.b, T)
    Th = _bcast(mech.Theta, T)
    return A * T[None] ** b * torch.exp(-Th / T[None])


def third_body_concentration(mech: MechT, C: torch.Tensor, j: int) -> torch.Tensor:
    """[M]_j = sum_s eps_sj C_s."""
    out = torch.zeros_like(C[0])
    for s in range(mech.ns):
        out = out + mech.efficiency[j, s] * C[s]
    return out


def troe_factor(mech: MechT, j: int, T: torch.Tensor, Pr: torch.Tensor) -> torch.Tensor:
    al, T3, T1, T2 = (float(x) for x in mech.troe[j])
    Fc = (1.0 - al) * torch.exp(-T / T3) + al * torch.exp(-T / T1) + torch.exp(-T2 / T)
    lFc = torch.log10(Fc)
    c = -0.4 - 0.67 * lFc
    n = 0.75 - 1.27 * lFc
    x = torch.log10(Pr) + c
    return 10.0 ** (lFc / (1.0 + (x / (n - 0.14 * x)) ** 2))


def effective_rate_factors(mech: MechT, C: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    """Per reaction the factor g_j multiplying the Arrhenius k_f in both directions:
    1 (elementary), [M]_j (third body) or P_r/(1 + P_r) F (fall-off)."""
    g = torch.ones((mech.nr,) + T.shape, dtype=T.dtype)
    if mech.rxn_type is None:
        return g
    for j in range(mech.nr):
        kind = int(mech.rxn_type[j])
        if kind == 0:
            continue
        M = third_body_concentration(mech, C, j)
        if kind == 1:
            g[j] = M
            continue
        kinf = mech.A[j] * T ** mech.b[j] * torch.exp(-mech.Theta[j] / T)
        k0 = mech.A0[j] * T ** mech.b0[j] * torch.exp(-mech.Theta0[j] / T)
        Pr = k0 * M / kinf
        F = troe_factor(mech, j, T, Pr) if kind == 3 else torch.ones_like(T)
        g[j] = Pr / (1.0 + Pr) * F
    return g


def equilibrium_constants(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """K_c [Nr, ...] in concentration units."""
    g = h_RT(mech, T) - s_R(mech, T)                 # [Ns, ...]
    dnu = mech.nu_r - mech.nu_f                      # [Nr, Ns]
    out = []
    for j in range(mech.nr):
        dg = torch.zeros_like(T)
        for s in range(mech.ns):
            if float(dnu[j, s]) != 0.0:
                dg = dg + dnu[j, s] * g[s]
        out.append(torch.exp(-dg) * (P_ATM / (R_U * T)) ** float(dnu[j].sum()))
    return torch.stack(out) if out else torch.zeros((0,) + T.shape, dtype=T.dtype)


def _conc_product(C: torch.Tensor, nu_row: torch.Tensor, skip: int = -1) -> torch.Tensor:
    """prod_s C_s^nu_s by repeated multiplication; `skip` removes one factor of C_skip."""
    out = torch.ones_like(C[0])
    for s in range(C.shape[0]):
        n = int(nu_row[s]) - (1 if s == skip else 0)
        for _ in range(n):
            out = out * C[s]
    return out


def rates_of_progress(mech: MechT, C: torch.Tensor, T: torch.Tensor):
    """Returns (q, forward term, reverse term), each [Nr, ...]."""
    kf = forward_rate_constants(mech, T) * effective_rate_factors(mech, C, T)
    Kc = equilibrium_constants(mech, T)
    fwd, rev = [], []
    for j in range(mech.nr):
        f = kf[j] * _conc_product(C, mech.nu_f[j])
        if bool(mech.reversible[j]):
            r = (kf[j] / Kc[j]) * _conc_product(C, mech.nu_r[j])
        else:
            r = torch.zeros_like(f)
        fwd.append(f)
        rev.append(r)
    if not fwd:
        z = torch.zeros((0,) + T.shape, dtype=T.dtype)
        return z, z, z
    fwd = torch.stack(fwd)
    rev = torch.stack(rev)
    return fwd - rev, fwd, rev


def production_rates(mech: MechT, rho_s: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    """omega_s [Ns, ...] in kg/m^3/s."""
    C = rho_s / _bcast(mech.W, T)
    q, _, _ = rates_of_progress(mech, C, T)
    dnu = mech.nu_r - mech.nu_f
    out = []
    for s in range(mech.ns):
        acc = torch.zeros_like(T)
        for j in range(mech.nr):
            if float(dnu[j, s]) != 0.0:
                acc = acc + dnu[j, s] * q[j]
        out.append(mech.W[s] * acc)
    return torch.stack(out)


def heat_release_rate(mech: MechT, omega: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    return -(species_h(mech, T) * omega).sum(0)


def chemical_rate(mech: MechT, rho_s: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    """max_s |d omega_s / d rho_s| at fixed T (diagonal of the chemical Jacobian),
    used by the time-step rule."""
    C = rho_s / _bcast(mech.W, T)
    kf = forward_rate_constants(mech, T) * effective_rate_factors(mech, C, T)
    Kc = equilibrium_constants(mech, T)
    dnu = mech.nu_r - mech.nu_f
    best = torch.zeros_like(T)
    for s in range(mech.ns):
        acc = torch.zeros_like(T)
        for j in range(mech.nr):
            if float(dnu[j, s]) == 0.0:
                continue
            d = torch.zeros_like(T)
            if float(mech.nu_f[j, s]) > 0:
                d = d + mech.nu_f[j, s] * kf[j] * _conc_product(C, mech.nu_f[j], skip=s)
            if bool(mech.reversible[j]) and float(mech.nu_r[j, s]) > 0:
                d = d - mech.nu_r[j, s] * (kf[j] / Kc[j]) * _conc_product(C, mech.nu_r[j], skip=s)
            acc = acc + dnu[j, s] * d
        best = torch.maximum(best, acc.abs())
    return best
