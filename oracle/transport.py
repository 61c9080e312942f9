"""Transport properties (Methods, Governing equations).

The paper evaluates the mixture viscosity by Wilke's rule, uses a mixture
thermal conductivity lambda in the heat flux, and a mixture-averaged
diffusivity D_s built from binary diffusivities.  The species laws below are
readings (the paper does not print them):

  mu_s     = mu_ref,s (T/300)^n_s
  lambda_s = mu_s (cp_s + 1.25 R / W_s)                      (modified Eucken)
  Phi_ij   = (1 + sqrt(mu_i/mu_j) (W_j/W_i)^(1/4))^2 / sqrt(8 (1 + W_i/W_j))
  mu       = sum_i X_i mu_i / sum_j X_j Phi_ij                (Wilke)
  lambda   = sum_i X_i lambda_i / sum_j X_j Phi_ij            (same Wilke form)
  D_ij     = D_ref,ij (T/300)^1.75 (p_atm / p)
  D_s      = sum_{j!=s} (X_j+eps) W_j / (Wbar_eps sum_{j!=s} (X_j+eps)/D_sj),
             Wbar_eps = sum_j (X_j+eps) W_j, eps = 1e-12
             (the (1 - Y_s) / sum_{j!=s} X_j / D_sj form, kept finite in pure streams);
             a one-species gas has D_1 = 0
"""
from __future__ import annotations

import torch

from .mech import P_ATM, R_U, MechT
from .thermo import _bcast

EPS_D = 1.0e-12


def species_viscosity(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    return _bcast(mech.mu_ref, T) * (T[None] / 300.0) ** _bcast(mech.mu_exp, T)


def species_conductivity(mech: MechT, mu_s: torch.Tensor, cp_s: torch.Tensor) -> torch.Tensor:
    return mu_s * (cp_s + 1.25 * _bcast(R_U / mech.W, mu_s[0]))


def wilke_phi(mech: MechT, mu_s: torch.Tensor) -> torch.Tensor:
    """Phi[i, j, ...]."""
    ns = mech.ns
    Wi = mech.W.reshape(ns, 1, *([1] * (mu_s.dim() - 1)))
    Wj = mech.W.reshape(1, ns, *([1] * (mu_s.dim() - 1)))
    mi = mu_s[:, None]
    mj = mu_s[None, :]
    return (1.0 + torch.sqrt(mi / mj) * (Wj / Wi) ** 0.25) ** 2 / torch.sqrt(8.0 * (1.0 + Wi / Wj))


def wilke_mixture(X: torch.Tensor, prop_s: torch.Tensor, phi: torch.Tensor) -> torch.Tensor:
    denom = (X[None, :] * phi).sum(1)          # sum_j X_j Phi_ij  -> [Ns, ...]
    return (X * prop_s / denom).sum(0)


def binary_diffusivity(mech: MechT, T: torch.Tensor, p: torch.Tensor) -> torch.Tensor:
    ns = mech.ns
    Dref = mech.D_ref.reshape(ns, ns, *([1] * T.dim()))
    return Dref * ((T / 300.0) ** 1.75 * (P_ATM / p))[None, None]


def mixture_diffusivity(mech: MechT, X: torch.Tensor, Dij: torch.Tensor) -> torch.Tensor:
    """D_s [Ns, ...]; a one-species gas has nothing to diffuse into and gets D = 0."""
    ns = mech.ns
    if ns == 1:
        return torch.zeros_like(X)
    Xe = X + EPS_D
    W = _bcast(mech.W, X[0])
    Wbar_eps = (Xe * W).sum(0)
    out = []
    for s in range(ns):
        num = torch.zeros_like(X[0])
        den = torch.zeros_like(X[0])
        for j in range(ns):
            if j == s:
                continue
            num = num + Xe[j] * W[j]
            den = den + Xe[j] / Dij[s, j]
        out.append(num / (Wbar_eps * den))
    return torch.stack(out)
