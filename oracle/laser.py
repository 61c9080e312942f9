"""Laser energy deposition (Methods, Diffusion flame: Eq. laser-qs).

The paper's source is a Gaussian in space and time,
  q_L = E_L / ((2 pi)^(3/2) sigma_r^2 sigma_t) exp(-r^2 / 2 sigma_r^2) exp(-(t-t0)^2 / 2 sigma_t^2),
with E_L an energy per unit depth of a two-dimensional domain.  Reading for
three-dimensional grids: the normalisation becomes (2 pi)^2 sigma_r^3 sigma_t,
so that the space-time integral of q_L equals E_L [J].  A grid with nz = 1 uses
the paper's two-dimensional form with r measured in the x-y plane.  Cell
centres sit at ((i + 1/2) dx, (j + 1/2) dy, (k + 1/2) dz) (on a mapped grid: the
mean of each cell's eight corners); no periodic images.
"""
from __future__ import annotations

import math

import torch


def cell_centres(grid, dtype=torch.float64):
    x = (torch.arange(grid.nx, dtype=dtype) + 0.5) * grid.dx
    y = (torch.arange(grid.ny, dtype=dtype) + 0.5) * grid.dy
    z = (torch.arange(grid.nz, dtype=dtype) + 0.5) * grid.dz
    Z, Y, X = torch.meshgrid(z, y, x, indexing="ij")
    return X, Y, Z


def laser_source(grid, t: float, las) -> torch.Tensor:
    """q_L [W/m^3] on the grid; `las` = (E, x0, y0, z0, sigma_r, t0, sigma_t),
    numbers or 0-d tensors."""
    E, x0, y0, z0, sr, t0, st = las
    if getattr(grid, "nodes", None) is not None:      # mapped grid: the cells' corner means
        from .mapped import cached_geometry
        X, Y, Z = cached_geometry(grid)["C"]
    else:
        X, Y, Z = cell_centres(grid)
    if grid.nz == 1:
        r2 = (X - x0) ** 2 + (Y - y0) ** 2
        norm = E / ((2.0 * math.pi) ** 1.5 * sr ** 2 * st)
    else:
        r2 = (X - x0) ** 2 + (Y - y0) ** 2 + (Z - z0) ** 2
        norm = E / ((2.0 * math.pi) ** 2 * sr ** 3 * st)
    tt = (t - t0) / st
    return norm * torch.exp(-0.5 * r2 / sr ** 2) * torch.exp(-0.5 * torch.as_tensor(tt, dtype=torch.float64) ** 2)
