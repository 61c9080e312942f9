"""Curvilinear (mapped) grids (Methods, Numerical method: the equations are
mapped from x-y-z onto a uniform xi-eta-zeta grid, U~ = U / J and
F~ = (xi_x F + xi_y G + xi_z H) / J and so on, and the Cartesian conservative
scheme is applied to the mapped fluxes; the fluxes are "mapped through covariant
transformation ... without sacrificing discrete conservation", after Vinokur 1974
and Pirozzoli 2011).  TEST INFRASTRUCTURE: the oracle's statement of the mapped
right-hand side.

The paper gives the mapped equations but not how the metric terms are
discretised.  Reading (a finite-volume-consistent evaluation that keeps a
uniform flow exactly uniform on any grid):
  * The grid is given by its node (cell corner) coordinates X[3, nz+1, ny+1, nx+1];
    the computational spacing is 1 along every axis.  Cell (i, j, k) has corners
    (i..i+1, j..j+1, k..k+1).
  * Metric of a face (xi_x/J, xi_y/J, xi_z/J for a face normal to xi, and so on):
    the face's area vector S = (d1 x d2) / 2 with d1, d2 the diagonals of its
    four corners, pointing towards increasing xi (eta, zeta).  The six area
    vectors of a cell sum to zero exactly (a closed surface), which is the
    discrete geometric conservation law; every face of every cell, the periodic
    seam included, takes its own corners.
  * 1/J of a cell (its volume): V = (1/3) sum over its six faces of the outward
    area vector dotted with the face centre (the mean of its corners).
  * Cell metric (the rows grad xi, grad eta, grad zeta): the inverse of the matrix
    whose columns are dx/dxi, dx/deta, dx/dzeta at the cell, each the mean of the
    cell's four edges along that axis.  Used for the viscous gradients (face
    value: the mean of the two cells) and the time-step rule.
  * Cell centre (laser position): the mean of the eight corners.
  * Inviscid flux through a face with area vector S, the metric frozen at the
    face: contravariant velocity theta = S . u, LLF speed
    alpha = max over the stencil of |theta| + c |S|, f+- = (theta U + p (0, S, theta)
    +- alpha U) / 2, reconstructed by WENO3-Z or TENO6 exactly as on a Cartesian
    grid; the WENO3-Z eps takes h = (V_L + V_R) / (2 |S|), the spacing normal to the
    face (h_x on a Cartesian grid).  A uniform state gives every face S . F(U)
    exactly, so the flux divergence of a uniform flow vanishes to rounding.
  * Diffusive flux through the face: physical gradients grad phi = sum_e
    (d phi / d xi_e) grad xi_e with the face metric the mean of the two cells'
    metrics, d/d xi along the face normal by the two-point difference and along
    the other axes by the mean of the two cells' central differences (the
    Cartesian face stencil with unit spacing); stress, heat and species-diffusion
    fluxes as on a Cartesian grid, dotted with S.
  * dU/dt = -sum of the face fluxes out of the cell / V + S_source.
On a uniform Cartesian grid every one of these reduces to the Cartesian scheme
(S = (dy dz, 0, 0) on x faces, V = dx dy dz, grad xi = (1/dx, 0, 0), ...).
"""
from __future__ import annotations

from dataclasses import dataclass

import torch

from . import fluxes
from .fluxes import NG, AX, cells, weno3z, teno6


@dataclass
class MappedGridT:
    nx: int
    ny: int
    nz: int
    nodes: torch.Tensor            # [3, nz+1, ny+1, nx+1] corner coordinates
    bc: tuple = (0, 0, 0)          # per axis: 0 periodic (in index space), 1 zero-gradient

    @property
    def n(self):
        return (self.nx, self.ny, self.nz)

    @property
    def h(self):
        return (1.0, 1.0, 1.0)      # computational spacing


def _cross(a, b):
    return torch.stack([a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]])


def geometry(grid: MappedGridT) -> dict:
    """Face area vectors S[d] ([3, faces of axis d]), cell volumes V, cell metric
    M[e, k] = d xi_e / d x_k ([3, 3, nz, ny, nx]) and cell centres C ([3, nz, ny, nx])."""
    X = grid.nodes.to(torch.float64)

    def P(i, j, k):
        """Corner (i + a, j + b, k + c) of every cell-sized slab: slices with
        offsets (0 or 1) along x, y, z; 'f' keeps the full face range."""
        sl = []
        for off, full in ((k, 2), (j, 1), (i, 0)):
            sl.append(slice(None) if off == "f" else slice(off, X.shape[1 + (2 - full)] - 1 + off))
        return X[(slice(None),) + tuple(sl)]

    # x faces: i in 0..nx (full), j, k cells
    Sx = 0.5 * _cross(P("f", 1, 1) - P("f", 0, 0), P("f", 0, 1) - P("f", 1, 0))
    cx = 0.25 * (P("f", 0, 0) + P("f", 1, 0) + P("f", 0, 1) + P("f", 1, 1))
    # y faces
    Sy = 0.5 * _cross(P(1, "f", 1) - P(0, "f", 0), P(1, "f", 0) - P(0, "f", 1))
    cy = 0.25 * (P(0, "f", 0) + P(1, "f", 0) + P(0, "f", 1) + P(1, "f", 1))
    # z faces
    Sz = 0.5 * _cross(P(1, 1, "f") - P(0, 0, "f"), P(0, 1, "f") - P(1, 0, "f"))
    cz = 0.25 * (P(0, 0, "f") + P(1, 0, "f") + P(0, 1, "f") + P(1, 1, "f"))

    def hi(f, d):
        return f.narrow(f.dim() + AX[d], 1, grid.n[d])

    def lo(f, d):
        return f.narrow(f.dim() + AX[d], 0, grid.n[d])
    flux = ((hi(Sx, 0) * hi(cx, 0)).sum(0) - (lo(Sx, 0) * lo(cx, 0)).sum(0)
            + (hi(Sy, 1) * hi(cy, 1)).sum(0) - (lo(Sy, 1) * lo(cy, 1)).sum(0)
            + (hi(Sz, 2) * hi(cz, 2)).sum(0) - (lo(Sz, 2) * lo(cz, 2)).sum(0))
    V = flux / 3.0
    # cell-centre derivatives of x along each computational axis: means of the 4 edges
    a_xi = 0.25 * ((P(1, 0, 0) - P(0, 0, 0)) + (P(1, 1, 0) - P(0, 1, 0))
                   + (P(1, 0, 1) - P(0, 0, 1)) + (P(1, 1, 1) - P(0, 1, 1)))
    a_eta = 0.25 * ((P(0, 1, 0) - P(0, 0, 0)) + (P(1, 1, 0) - P(1, 0, 0))
                    + (P(0, 1, 1) - P(0, 0, 1)) + (P(1, 1, 1) - P(1, 0, 1)))
    a_zeta = 0.25 * ((P(0, 0, 1) - P(0, 0, 0)) + (P(1, 0, 1) - P(1, 0, 0))
                     + (P(0, 1, 1) - P(0, 1, 0)) + (P(1, 1, 1) - P(1, 1, 0)))
    A = torch.stack([a_xi, a_eta, a_zeta], dim=1)           # A[k, e] = d x_k / d xi_e
    Ai = torch.linalg.inv(A.permute(2, 3, 4, 0, 1))         # [..., e, k] = d xi_e / d x_k
    M = Ai.permute(3, 4, 0, 1, 2).contiguous()
    C = 0.125 * sum(P(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1))
    return {"S": [Sx, Sy, Sz], "V": V, "M": M, "C": C}


def euler_flux_S(U, vel, p, S, ns):
    """S . (F, G, H) of the state U: theta U + p (0, S, theta), theta = S . u."""
    theta = S[0] * vel[0] + S[1] * vel[1] + S[2] * vel[2]
    F = theta[None] * U
    F = F.clone()
    for k in range(3):
        F[ns + k] = F[ns + k] + p * S[k]
    F[ns + 3] = F[ns + 3] + p * theta
    return F, theta


def inviscid_flux(Up, velp, pp, cp, Vp, S, grid, d, ns, scheme="weno3z"):
    """LLF-split flux through every face of axis d, the metric frozen at the face."""
    offs = (-3, -2, -1, 0, 1, 2) if scheme == "teno6" else (-2, -1, 0, 1)
    Smag = torch.sqrt(S[0] ** 2 + S[1] ** 2 + S[2] ** 2)
    Us = {o: cells(Up, grid, d, o) for o in offs}
    vs = {o: [cells(velp[k], grid, d, o) for k in range(3)] for o in offs}
    ps = {o: cells(pp, grid, d, o) for o in offs}
    cs = {o: cells(cp, grid, d, o) for o in offs}
    Fs, th = {}, {}
    for o in offs:
        Fs[o], th[o] = euler_flux_S(Us[o], vs[o], ps[o], S, ns)
    alpha = None
    for o in offs:
        lam = th[o].abs() + cs[o] * Smag
        alpha = lam if alpha is None else torch.maximum(alpha, lam)
    fp = {o: 0.5 * (Fs[o] + alpha[None] * Us[o]) for o in offs}
    fm = {o: 0.5 * (Fs[o] - alpha[None] * Us[o]) for o in offs}
    if scheme == "teno6":
        return teno6([fp[o] for o in offs]) + teno6([fm[o] for o in reversed(offs)])
    h = 0.5 * (cells(Vp, grid, d, -1) + cells(Vp, grid, d, 0)) / Smag
    return weno3z(fp[-2], fp[-1], fp[0], h) + weno3z(fm[1], fm[0], fm[-1], h)


def diffusive_flux(velp, Tp, Xp, Yp, Dcp, hp, mup, lamp, Mp, S, grid, d, ns):
    """Viscous + heat-conduction + species-diffusion flux through every face of axis d."""
    def avg(P):
        return 0.5 * (cells(P, grid, d, -1) + cells(P, grid, d, 0))

    def dxi(P, e):
        if e == d:
            return cells(P, grid, d, 0) - cells(P, grid, d, -1)
        left = cells(P, grid, d, -1, {e: 1}) - cells(P, grid, d, -1, {e: -1})
        right = cells(P, grid, d, 0, {e: 1}) - cells(P, grid, d, 0, {e: -1})
        return 0.25 * (left + right)

    Mf = avg(Mp)                                            # [3 e, 3 k, faces]

    def grad(P):
        """[3 k, ...] physical gradient of P at the faces (P may carry a leading axis)."""
        g = [dxi(P, e) for e in range(3)]
        if P.dim() == 4:
            return torch.stack([sum(g[e] * Mf[e, k][None] for e in range(3)) for k in range(3)])
        return torch.stack([sum(g[e] * Mf[e, k] for e in range(3)) for k in range(3)])

    mu = avg(mup)
    lam = avg(lamp)
    uf = [avg(velp[m]) for m in range(3)]
    gu = [grad(velp[l]) for l in range(3)]                  # gu[l][k] = d u_l / d x_k
    div = gu[0][0] + gu[1][1] + gu[2][2]
    tau = [[mu * (gu[l][k] + gu[k][l]) - ((2.0 / 3.0) * mu * div if k == l else 0.0) for l in range(3)]
           for k in range(3)]
    gX = grad(Xp)                                           # [3 k, ns, faces]
    Dc = avg(Dcp)
    Yf = avg(Yp)
    hf = avg(hp)
    J = []
    for k in range(3):
        jd = Dc * gX[k]
        J.append(-jd + Yf * jd.sum(0)[None])
    gT = grad(Tp)
    q = [-lam * gT[k] + (J[k] * hf).sum(0) for k in range(3)]
    out = [-(J[0][s] * S[0] + J[1][s] * S[1] + J[2][s] * S[2]) for s in range(ns)]
    for l in range(3):
        out.append(S[0] * tau[0][l] + S[1] * tau[1][l] + S[2] * tau[2][l])
    work = [tau[k][0] * uf[0] + tau[k][1] * uf[1] + tau[k][2] * uf[2] for k in range(3)]
    out.append(sum(S[k] * (work[k] - q[k]) for k in range(3)))
    return torch.stack(out)


def divergence(F, grid, d, V):
    """(F_{f+1} - F_f) / V over the cells of axis d."""
    n = grid.n[d]
    ax = F.dim() + AX[d]
    return (F.narrow(ax, 1, n) - F.narrow(ax, 0, n)) / V


def cached_geometry(grid) -> dict:
    geo = getattr(grid, "_geometry", None)
    if geo is None:
        geo = geometry(grid)
        object.__setattr__(grid, "_geometry", geo)
    return geo


def rate_limits(grid, st):
    """Per-cell acoustic rate sum_e (|u . grad xi_e| + c |grad xi_e|) and the factor
    max_e |grad xi_e|^2 of the diffusive limit, over the axes with more than one cell."""
    M = cached_geometry(grid)["M"]
    ac = torch.zeros_like(st["T"])
    g2 = torch.zeros_like(st["T"])
    for e in range(3):
        if grid.n[e] <= 1:
            continue
        un = M[e, 0] * st["vel"][0] + M[e, 1] * st["vel"][1] + M[e, 2] * st["vel"][2]
        m2 = M[e, 0] ** 2 + M[e, 1] ** 2 + M[e, 2] ** 2
        ac = ac + un.abs() + st["c"] * torch.sqrt(m2)
        g2 = torch.maximum(g2, m2)
    return ac, g2
