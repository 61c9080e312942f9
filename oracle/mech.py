"""Mechanism and grid containers for the oracle (float64 CPU tensors)."""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import torch

R_U = 8.314462618        # universal gas constant, J/mol/K
P_ATM = 101325.0         # standard-state pressure, Pa
DT = torch.float64


@dataclass
class MechT:
    W: torch.Tensor          # [Ns] kg/mol
    elem: torch.Tensor       # [Ns, Ne]
    nasa_low: torch.Tensor   # [Ns, 7]
    nasa_high: torch.Tensor  # [Ns, 7]
    T_mid: torch.Tensor      # [Ns]
    mu_ref: torch.Tensor     # [Ns]
    mu_exp: torch.Tensor     # [Ns]
    D_ref: torch.Tensor      # [Ns, Ns]
    A: torch.Tensor          # [Nr] SI
    b: torch.Tensor          # [Nr]
    Theta: torch.Tensor      # [Nr] K
    nu_f: torch.Tensor       # [Nr, Ns] (float)
    nu_r: torch.Tensor       # [Nr, Ns] (float)
    reversible: torch.Tensor  # [Nr] bool

    @property
    def ns(self) -> int:
        return int(self.W.shape[0])

    @property
    def nr(self) -> int:
        return int(self.A.shape[0])

    def with_A(self, A: torch.Tensor) -> "MechT":
        d = dict(self.__dict__)
        d["A"] = A
        return MechT(**d)


@dataclass
class GridT:
    nx: int
    ny: int
    nz: int
    dx: float
    dy: float
    dz: float
    bc: tuple = (0, 0, 0)     # per axis x, y, z: 0 periodic, 1 zero-gradient extrapolation

    @property
    def n(self):
        return (self.nx, self.ny, self.nz)

    @property
    def h(self):
        return (self.dx, self.dy, self.dz)


def from_synth(m) -> MechT:
    t = lambda a: torch.as_tensor(a, dtype=DT).clone()
    return MechT(W=t(m.W), elem=t(m.elem), nasa_low=t(m.nasa_low), nasa_high=t(m.nasa_high),
                 T_mid=t(m.T_mid), mu_ref=t(m.mu_ref), mu_exp=t(m.mu_exp), D_ref=t(m.D_ref),
                 A=t(m.A), b=t(m.b), Theta=t(m.Theta), nu_f=t(m.nu_f), nu_r=t(m.nu_r),
                 reversible=torch.as_tensor(m.reversible).bool())


def grid_from_synth(g) -> GridT:
    return GridT(g.nx, g.ny, g.nz, float(g.dx), float(g.dy), float(g.dz), tuple(int(b) for b in g.bc))
