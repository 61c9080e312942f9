"""Thermodynamics: NASA polynomials, ideal-gas EOS, temperature recovery.

Follows Methods, Governing equations: the ideal-gas equation of state
p = rho R T sum_s Y_s / W_s, and species heat capacities from NASA
polynomial fits.

Readings (the paper names nine-coefficient NASA fits; the workloads use the
seven-coefficient form):
  * NASA-7, two ranges split at T_mid per species:
      cp/R = a1 + a2 T + a3 T^2 + a4 T^3 + a5 T^4
      h/RT = a1 + a2 T/2 + a3 T^2/3 + a4 T^3/4 + a5 T^4/5 + a6/T
      s/R  = a1 ln T + a2 T + a3 T^2/2 + a4 T^3/3 + a5 T^4/4 + a7
    h includes the formation enthalpy, so the total energy E carries the
    chemical energy and chemistry adds no source to E.
  * Temperature from the specific internal energy e = sum_s Y_s e_s(T),
    e_s = h_s - R T / W_s, by Newton's method warm-started from the stored T:
    T <- T - (e(T) - e) / cv(T) until |dT| <= 1e-13 T, at most 30 iterations;
    no clipping of T.
  * Frozen speed of sound c = sqrt(gamma p / rho), gamma = cp / (cp - R/Wbar).
"""
from __future__ import annotations

import torch

from .mech import R_U, MechT


def _bcast(v: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    """Per-species vector -> shape [Ns, 1, ..., 1] broadcastable against T[None]."""
    return v.reshape(v.shape + (1,) * T.dim())


def coefficients(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """NASA-7 coefficients of the range containing T: [Ns, 7, *T.shape]."""
    low = mech.nasa_low.reshape(mech.ns, 7, *([1] * T.dim()))
    high = mech.nasa_high.reshape(mech.ns, 7, *([1] * T.dim()))
    use_low = (T[None] < _bcast(mech.T_mid, T))[:, None]
    return torch.where(use_low, low, high)


def cp_R(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    a = coefficients(mech, T)
    return a[:, 0] + a[:, 1] * T + a[:, 2] * T ** 2 + a[:, 3] * T ** 3 + a[:, 4] * T ** 4


def h_RT(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    a = coefficients(mech, T)
    return (a[:, 0] + a[:, 1] * T / 2 + a[:, 2] * T ** 2 / 3 + a[:, 3] * T ** 3 / 4
            + a[:, 4] * T ** 4 / 5 + a[:, 5] / T)


def s_R(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    a = coefficients(mech, T)
    return (a[:, 0] * torch.log(T) + a[:, 1] * T + a[:, 2] * T ** 2 / 2 + a[:, 3] * T ** 3 / 3
            + a[:, 4] * T ** 4 / 4 + a[:, 6])


def species_cp(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """cp_s [J/kg/K], shape [Ns, *T.shape]."""
    return cp_R(mech, T) * _bcast(R_U / mech.W, T)


def species_h(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """h_s [J/kg] including formation enthalpy."""
    return h_RT(mech, T) * R_U * T / _bcast(mech.W, T)


def species_e(mech: MechT, T: torch.Tensor) -> torch.Tensor:
    """e_s = h_s - R T / W_s [J/kg]."""
    return (h_RT(mech, T) - 1.0) * R_U * T / _bcast(mech.W, T)


def mean_molar_mass(mech: MechT, Y: torch.Tensor) -> torch.Tensor:
    """Wbar = 1 / sum_s Y_s / W_s."""
    return 1.0 / (Y / _bcast(mech.W, Y[0])).sum(0)


def pressure(mech: MechT, rho: torch.Tensor, Y: torch.Tensor, T: torch.Tensor) -> torch.Tensor:
    """Ideal-gas EOS p = rho R T sum_s Y_s / W_s."""
    return rho * R_U * T * (Y / _bcast(mech.W, T)).sum(0)


def temperature_from_energy(mech: MechT, Y: torch.Tensor, e: torch.Tensor, T0: torch.Tensor,
                            tol: float = 1.0e-13, maxit: int = 30):
    """Newton solve of sum_s Y_s e_s(T) = e.  Returns (T, converged, iterations).

    Each cell iterates until its own update satisfies |dT| <= tol * T; a cell
    that has converged is not updated again."""
    T = T0.clone()
    done = torch.zeros_like(T, dtype=torch.bool)
    its = torch.zeros_like(T, dtype=torch.int32)
    for _ in range(maxit):
        if bool(done.all()):
            break
        em = (Y * species_e(mech, T)).sum(0)
        cv = (Y * (species_cp(mech, T) - _bcast(R_U / mech.W, T))).sum(0)
        dT = (em - e) / cv
        Tn = T - dT
        T = torch.where(done, T, Tn)
        its = its + (~done).to(torch.int32)
        done = done | (dT.abs() <= tol * Tn.abs())
    return T, done, its


def sound_speed(mech: MechT, rho, p, Y, T, Wbar):
    cp = (Y * species_cp(mech, T)).sum(0)
    gamma = cp / (cp - R_U / Wbar)
    return torch.sqrt(gamma * p / rho)
