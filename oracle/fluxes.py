"""Inviscid and diffusive face fluxes (Methods, Numerical method).

The paper discretises the Cartesian-grid conservation law
  dU/dt + dF^a/dx + dG^a/dy + dH^a/dz = dF^d/dx + dG^d/dy + dH^d/dz + S
with a conservative finite-difference method: WENO3-Z (or TENO6) for the
inviscid fluxes under a flux splitting, and second-order central differences
for the diffusive fluxes.  On the uniform Cartesian grids used here the metric
terms of the curvilinear form are the identity.

Readings:
  * Inviscid: component-wise local Lax-Friedrichs splitting of the conserved
    variables, f^(+-)_m = (F(U_m) +- alpha U_m) / 2, with
    alpha_{i+1/2} = max_{m = i-1..i+2} (|u_n,m| + c_m); the face flux is
    WENO3-Z(f^+ from cells i-1, i, i+1) + WENO3-Z(f^- mirrored, cells i+2, i+1, i).
  * WENO3-Z at i+1/2 from (a, b, c) = (f_{i-1}, f_i, f_{i+1}):
      q0 = -a/2 + 3b/2, q1 = b/2 + c/2, beta0 = (b-a)^2, beta1 = (c-b)^2,
      tau = |beta1 - beta0|, alpha_k = d_k (1 + tau / (beta_k + eps)),
      d = (1/3, 2/3), eps = 1e-30, result = (alpha0 q0 + alpha1 q1) / (alpha0 + alpha1),
      evaluated as q1 + omega0 (q0 - q1) (see weno3z).
  * Diffusive, at the face between cells L and R: normal derivatives by the
    two-point difference, tangential derivatives by the mean of the two cells'
    central differences, coefficients by arithmetic means.  Stokes hypothesis,
    no Soret or Dufour terms.
      J_s   = -Dc_s dX_s/dn + Y_s sum_k Dc_k dX_k/dn,  Dc_s = rho D_s W_s / Wbar
      tau   = mu (grad u + grad u^T) - (2/3) mu (div u) I
      q     = -lambda dT/dn + sum_s J_s h_s
    fluxes: species -J_s, momentum tau . n, energy (tau . u) . n - q.
  * Ghost cells: periodic axes wrap, zero-gradient axes copy the edge cell.
"""
from __future__ import annotations

import torch

NG = 2
EPS_WENO = 1.0e-30
AX = (-1, -2, -3)        # tensor axis of x, y, z


def pad(f: torch.Tensor, grid) -> torch.Tensor:
    """Add NG ghost layers on every side of the three trailing (z, y, x) axes."""
    out = f
    for a in range(3):
        n = grid.n[a]
        i = torch.arange(-NG, n + NG)
        if grid.bc[a] == 0:
            idx = torch.remainder(i, n)
        else:
            idx = torch.clamp(i, 0, n - 1)
        out = out.index_select(out.dim() + AX[a], idx)
    return out


def cells(P: torch.Tensor, grid, d: int, off: int, tan: dict | None = None) -> torch.Tensor:
    """Values at cells f + off for every face f = 0..n_d of axis d (face f lies
    between cells f-1 and f), interior cells along the other axes, shifted by
    tan[a] along tangential axis a."""
    idx = [slice(None)] * P.dim()
    for a in range(3):
        n = grid.n[a]
        if a == d:
            idx[P.dim() + AX[a]] = slice(NG + off, NG + off + n + 1)
        else:
            o = tan.get(a, 0) if tan else 0
            idx[P.dim() + AX[a]] = slice(NG + o, NG + o + n)
    return P[tuple(idx)]


def weno3z(a, b, c):
    """Upwind-biased WENO3-Z value at i+1/2 from (f_{i-1}, f_i, f_{i+1}).

    The weighted sum omega0 q0 + omega1 q1 is written q1 + omega0 (q0 - q1), the
    same value since omega0 + omega1 = 1, with q0 - q1 = ((b - a) - (c - b)) / 2:
    reverse-mode derivatives of the weights then multiply differences of f, not
    values of f, and stay accurate where f varies by far less than its size."""
    q1 = 0.5 * b + 0.5 * c
    beta0 = (b - a) ** 2
    beta1 = (c - b) ** 2
    tau = (beta1 - beta0).abs()
    alpha0 = (1.0 / 3.0) * (1.0 + tau / (beta0 + EPS_WENO))
    alpha1 = (2.0 / 3.0) * (1.0 + tau / (beta1 + EPS_WENO))
    omega0 = alpha0 / (alpha0 + alpha1)
    return q1 + omega0 * (0.5 * ((b - a) - (c - b)))


def euler_flux(U: torch.Tensor, vel, p: torch.Tensor, d: int, ns: int) -> torch.Tensor:
    """F(U) along axis d: u_d U + p (momentum d) + p u_d (energy)."""
    un = vel[d]
    F = un[None] * U
    F = F.clone()
    F[ns + d] = F[ns + d] + p
    F[ns + 3] = F[ns + 3] + p * un
    return F


def inviscid_flux(Up, velp, pp, cp, grid, d: int, ns: int) -> torch.Tensor:
    """LLF-split WENO3-Z numerical flux at every face of axis d: [nv, faces...]."""
    offs = (-2, -1, 0, 1)
    Us = {o: cells(Up, grid, d, o) for o in offs}
    vs = {o: [cells(velp[k], grid, d, o) for k in range(3)] for o in offs}
    ps = {o: cells(pp, grid, d, o) for o in offs}
    cs = {o: cells(cp, grid, d, o) for o in offs}
    alpha = None
    for o in offs:
        lam = vs[o][d].abs() + cs[o]
        alpha = lam if alpha is None else torch.maximum(alpha, lam)
    Fs = {o: euler_flux(Us[o], vs[o], ps[o], d, ns) for o in offs}
    fp = {o: 0.5 * (Fs[o] + alpha[None] * Us[o]) for o in offs}
    fm = {o: 0.5 * (Fs[o] - alpha[None] * Us[o]) for o in offs}
    return weno3z(fp[-2], fp[-1], fp[0]) + weno3z(fm[1], fm[0], fm[-1])


def diffusive_flux(velp, Tp, Xp, Yp, Dcp, hp, mup, lamp, grid, d: int, ns: int) -> torch.Tensor:
    """Viscous + heat-conduction + species-diffusion flux at every face of axis d."""
    h = grid.h

    def avg(P):
        return 0.5 * (cells(P, grid, d, -1) + cells(P, grid, d, 0))

    def dn(P):
        return (cells(P, grid, d, 0) - cells(P, grid, d, -1)) / h[d]

    def dt_(P, t):
        left = cells(P, grid, d, -1, {t: 1}) - cells(P, grid, d, -1, {t: -1})
        right = cells(P, grid, d, 0, {t: 1}) - cells(P, grid, d, 0, {t: -1})
        return 0.5 * (left + right) / (2.0 * h[t])

    def grad(P, m):
        return dn(P) if m == d else dt_(P, m)

    mu = avg(mup)
    lam = avg(lamp)
    uf = [avg(velp[m]) for m in range(3)]
    div = grad(velp[0], 0) + grad(velp[1], 1) + grad(velp[2], 2)
    tau = []
    for m in range(3):
        t = mu * (grad(velp[d], m) + dn(velp[m]))
        if m == d:
            t = t - (2.0 / 3.0) * mu * div
        tau.append(t)
    dX = dn(Xp)
    Dc = avg(Dcp)
    Yf = avg(Yp)
    hf = avg(hp)
    corr = (Dc * dX).sum(0)
    J = -Dc * dX + Yf * corr[None]
    q = -lam * dn(Tp) + (J * hf).sum(0)
    out = [-J[s] for s in range(ns)]
    out += tau
    out.append(tau[0] * uf[0] + tau[1] * uf[1] + tau[2] * uf[2] - q)
    return torch.stack(out)


def divergence(F: torch.Tensor, grid, d: int) -> torch.Tensor:
    """(F_{f+1} - F_f) / h_d over the cells of axis d."""
    n = grid.n[d]
    ax = F.dim() + AX[d]
    hi = F.narrow(ax, 1, n)
    lo = F.narrow(ax, 0, n)
    return (hi - lo) / grid.h[d]
