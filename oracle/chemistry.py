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
"""
from __future__ import annotations

import torch

from .mech import P_ATM, R_U, MechT
from .thermo import _bcast, h_RT, s_R, species_h


def forward_rate_constants(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """k_f [Nr, ...]."""
    A = _bcast(mech.A, T)
    b = _bcast(mech.b, T)
    Th = _bcast(mech.Theta, T)
    return A * T[None] ** b * torch.exp(-Th / T[None])


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
    kf = forward_rate_constants(mech, T)
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
    kf = forward_rate_constants(mech, T)
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
