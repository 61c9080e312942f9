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
    # pressure-dependent reactions (None: all elementary): type [Nr] 0 elementary,
    # 1 third body, 2 Lindemann, 3 Troe; efficiencies [Nr, Ns]; low-pressure
    # Arrhenius A0, b0, Theta0 [Nr]; Troe alpha, T***, T*, T** [Nr, 4]
    rxn_type: Optional[torch.Tensor] = None
    efficiency: Optional[torch.Tensor] = None
    A0: Optional[torch.Tensor] = None
    b0: Optional[torch.Tensor] = None
    Theta0: Optional[torch.Tensor] = None
    troe: Optional[torch.Tensor] = None

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
    bc: tuple = (0, 0, 0)     # per axis x, y, z: 0 periodic, 1 zero-gradient extrapolation, 2 NSCBC

    @property
    def n(self):
        return (self.nx, self.ny, self.nz)

    @property
    def h(self):
        return (self.dx, self.dy, self.dz)


def from_synth(m) -> MechT:
    t = lambda a: torch.as_tensor(a, dtype=DT).clone()
    opt = lambda a: None if a is None else t(a)
    rt = getattr(m, "rxn_type", None)
    return MechT(W=t(m.W), elem=t(m.elem), nasa_low=t(m.nasa_low), nasa_high=t(m.nasa_high),
                 T_mid=t(m.T_mid), mu_ref=t(m.mu_ref), mu_exp=t(m.mu_exp), D_ref=t(m.D_ref),
                 A=t(m.A), b=t(m.b), Theta=t(m.Theta), nu_f=t(m.nu_f), nu_r=t(m.nu_r),
                 reversible=torch.as_tensor(m.reversible).bool(),
                 rxn_type=None if rt is None else torch.as_tensor(rt, dtype=torch.int64).clone(),
                 efficiency=opt(getattr(m, "efficiency", None)), A0=opt(getattr(m, "A0", None)),
                 b0=opt(getattr(m, "b0", None)), Theta0=opt(getattr(m, "Theta0", None)),
                 troe=opt(getattr(m, "troe", None)))


def grid_from_synth(g) -> GridT:
    return GridT(g.nx, g.ny, g.nz, float(g.dx), float(g.dy), float(g.dz), tuple(int(b) for b in g.bc))
