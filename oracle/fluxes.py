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
      d = (1/3, 2/3), result = (alpha0 q0 + alpha1 q1) / (alpha0 + alpha1),
      evaluated as q1 + omega0 (q0 - q1) (see weno3z).  The paper leaves eps open;
      reading: the grid-scaled eps = h^2 (a^2 + b^2 + c^2) / 3 + 1e-30, h the grid
      spacing along the sweep (in the problem's length unit).  An eps of order h^2
      restores third order at smooth extrema, where a fixed tiny eps lets the Z
      weights drop to second order (the remedy published for WENO-Z at critical
      points); scaling it by the mean square of the three values makes the weights
      independent of each variable's units, and 1e-30 keeps it positive where all
      three values vanish.
  * TENO6 (the paper's other scheme, after Fu, Hu and Adams, J. Comput. Phys. 305
    (2016)), at i+1/2 from f_{i-2} .. f_{i+3}: candidate stencils S0 = {i-1, i, i+1},
    S1 = {i, i+1, i+2}, S2 = {i-2, i-1, i}, S3 = {i, i+1, i+2, i+3}, each with the
    value q_k at i+1/2 of the polynomial whose cell averages are the f_j of the
    stencil and the Jiang-Shu smoothness indicator
      beta = sum_{l >= 1} h^(2l-1) int_{x_{i-1/2}}^{x_{i+1/2}} (d^l p / dx^l)^2 dx;
    d = (9, 6, 1, 4) / 20 (the weights that make sum d_k q_k the six-point value);
    tau = |beta_6 - (beta_1 + beta_2 + 4 beta_0) / 6| with beta_6 the indicator of the
    whole six-point stencil; gamma_k = (1 + tau / (beta_k + eps))^6, chi_k = gamma_k /
    sum gamma; stencil k is kept (delta_k = 1) if chi_k >= C_T, else dropped; the value
    is sum d_k delta_k q_k / sum d_k delta_k.  Readings: C_T = 1e-7, eps = 1e-30 (as for
    WENO3-Z: representable in FP32), and the LLF alpha the maximum over the six cells.
    The polynomials, candidate values and indicators are built here from their
    definitions (exact rational arithmetic); see teno6.
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

from fractions import Fraction

import torch

NG = 3
EPS_WENO = 1.0e-30
TENO_CT = 1.0e-7
TENO_EPS = 1.0e-30
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


def weno3z(a, b, c, h):
    """Upwind-biased WENO3-Z value at i+1/2 from (f_{i-1}, f_i, f_{i+1}), grid
    spacing h along the reconstruction.

    The weighted sum omega0 q0 + omega1 q1 is written q1 + omega0 (q0 - q1), the
    same value since omega0 + omega1 = 1, with q0 - q1 = ((b - a) - (c - b)) / 2:
    reverse-mode derivatives of the weights then multiply differences of f, not
    values of f, and stay accurate where f varies by far less than its size."""
    return weno3z_eps(a, b, c, h * h * (a * a + b * b + c * c) / 3.0 + EPS_WENO)


def weno3z_eps(a, b, c, eps):
    """WENO3-Z value at i+1/2 with a given eps (see weno3z)."""
    q1 = 0.5 * b + 0.5 * c
    beta0 = (b - a) ** 2
    beta1 = (c - b) ** 2
    tau = (beta1 - beta0).abs()
    alpha0 = (1.0 / 3.0) * (1.0 + tau / (beta0 + eps))
    alpha1 = (2.0 / 3.0) * (1.0 + tau / (beta1 + eps))
    omega0 = alpha0 / (alpha0 + alpha1)
    return q1 + omega0 * (0.5 * ((b - a) - (c - b)))


def _solve_exact(A, b):
    """Solve A x = b for square rational A (Gauss-Jordan on Fractions)."""
    n = len(A)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        pv = M[c][c]
        M[c] = [v / pv for v in M[c]]
        for r in range(n):
            if r != c and M[r][c] != 0:
                fac = M[r][c]
                M[r] = [vr - fac * vc for vr, vc in zip(M[r], M[c])]
    return [M[i][n] for i in range(n)]


def _mono_int(k, lo, hi):
    """Integral of x^k over [lo, hi]."""
    return (hi ** (k + 1) - lo ** (k + 1)) / (k + 1)


def stencil_forms(offsets):
    """For the stencil of cells i + o (o in offsets, unit spacing, x = 0 the centre
    of cell i): the polynomial p with the cell averages f_{i+o} has coefficients
    c = C f; returns (w, B) with p(1/2) = w . f (the value at i+1/2) and the
    Jiang-Shu indicator sum_{l>=1} int_{-1/2}^{1/2} (p^(l))^2 dx = f^T B f, both exact
    rationals (the indicator of a uniform grid does not depend on h)."""
    n = len(offsets)
    half = Fraction(1, 2)
    A = [[_mono_int(k, Fraction(o) - half, Fraction(o) + half) for k in range(n)] for o in offsets]
    # columns of C: the coefficients of p for a unit value in each cell
    cols = [_solve_exact(A, [Fraction(int(j == m)) for j in range(n)]) for m in range(n)]
    C = [[cols[m][k] for m in range(n)] for k in range(n)]          # C[k][m]
    w = [sum(C[k][m] * half ** k for k in range(n)) for m in range(n)]
    # d^l/dx^l x^k = k!/(k-l)! x^(k-l); int_{-1/2}^{1/2} x^(a+b) dx
    def fall(k, l):
        out = 1
        for t in range(l):
            out *= (k - t)
        return out
    Q = [[sum(fall(a, l) * fall(b, l) * _mono_int(a + b - 2 * l, -half, half)
              for l in range(1, n) if a >= l and b >= l) for b in range(n)] for a in range(n)]
    B = [[sum(C[a][m1] * Q[a][b] * C[b][m2] for a in range(n) for b in range(n)) for m2 in range(n)]
         for m1 in range(n)]
    return w, B


def sum_of_squares(B):
    """The positive semidefinite rational form f^T B f as sum_k d_k (L_k . f)^2 with
    d_k > 0 (an exact LDL^T factorisation), so that it cannot round below zero."""
    n = len(B)
    L = [[Fraction(0)] * n for _ in range(n)]
    d = [Fraction(0)] * n
    for k in range(n):
        d[k] = B[k][k] - sum(L[k][j] ** 2 * d[j] for j in range(k))
        if d[k] == 0:
            continue
        L[k][k] = Fraction(1)
        for i in range(k + 1, n):
            L[i][k] = (B[i][k] - sum(L[i][j] * L[k][j] * d[j] for j in range(k))) / d[k]
    return [(d[k], [L[i][k] for i in range(n)]) for k in range(n) if d[k] != 0]


# TENO6 stencils as offsets from cell i (the face is i+1/2), in the order S0 .. S3,
# then the whole six-point stencil
TENO6_STENCILS = ((-1, 0, 1), (0, 1, 2), (-2, -1, 0), (0, 1, 2, 3), (-2, -1, 0, 1, 2, 3))
_TENO6_FORMS = [stencil_forms(o) for o in TENO6_STENCILS]


def _sixpoint_weights():
    """d_k with sum_k d_k q_k = the six-point value (exact)."""
    w6 = _TENO6_FORMS[4][0]
    # unknowns d0..d3; match the coefficients of f_{i-2} .. f_{i+3}
    rows, rhs = [], []
    for j, o in enumerate(TENO6_STENCILS[4]):
        row = []
        for k in range(4):
            offs = TENO6_STENCILS[k]
            row.append(_TENO6_FORMS[k][0][offs.index(o)] if o in offs else Fraction(0))
        rows.append(row)
        rhs.append(w6[j])
    # six equations, four unknowns: solve the first four independent ones, check all
    d = _solve_exact([rows[0], rows[5], rows[1], rows[4]], [rhs[0], rhs[5], rhs[1], rhs[4]])
    for r, v in zip(rows, rhs):
        assert sum(a * b for a, b in zip(r, d)) == v
    return d


TENO6_D = _sixpoint_weights()
_TENO6_SQUARES = [sum_of_squares(B) for _, B in _TENO6_FORMS]


def teno6(f, C_T: float = TENO_CT):
    """TENO6 value at i+1/2 from f = (f_{i-2}, f_{i-1}, f_i, f_{i+1}, f_{i+2}, f_{i+3})
    (tensors of equal shape); see the module docstring."""
    base = -2
    q, beta = [], []
    for k, offs in enumerate(TENO6_STENCILS):
        w, _ = _TENO6_FORMS[k]
        fk = [f[o - base] for o in offs]
        if k < 4:
            q.append(sum(float(w[m]) * fk[m] for m in range(len(offs))))
        beta.append(sum(float(dk) * sum(float(c) * v for c, v in zip(Lk, fk)) ** 2 for dk, Lk in _TENO6_SQUARES[k]))
    tau = (beta[4] - (beta[1] + beta[2] + 4.0 * beta[0]) / 6.0).abs()
    # gamma_k = (1 + tau / (beta_k + eps))^6 and chi_k = gamma_k / sum gamma, formed
    # from logarithms so that no gamma overflows
    lg = torch.stack([6.0 * torch.log1p(tau / (beta[k] + TENO_EPS)) for k in range(4)])
    chi = torch.softmax(lg, dim=0)
    keep = (chi >= C_T).to(f[0].dtype)
    num = sum(float(TENO6_D[k]) * keep[k] * q[k] for k in range(4))
    den = sum(float(TENO6_D[k]) * keep[k] for k in range(4))
    return num / den


def euler_flux(U: torch.Tensor, vel, p: torch.Tensor, d: int, ns: int) -> torch.Tensor:
    """F(U) along axis d: u_d U + p (momentum d) + p u_d (energy)."""
    un = vel[d]
    F = un[None] * U
    F = F.clone()
    F[ns + d] = F[ns + d] + p
    F[ns + 3] = F[ns + 3] + p * un
    return F


def inviscid_flux(Up, velp, pp, cp, grid, d: int, ns: int, scheme: str = "weno3z") -> torch.Tensor:
    """LLF-split numerical flux (WENO3-Z, or TENO6) at every face of axis d: [nv, faces...]."""
    if scheme == "teno6":
        return _inviscid_flux_teno6(Up, velp, pp, cp, grid, d, ns)
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
    h = grid.h[d]
    return weno3z(fp[-2], fp[-1], fp[0], h) + weno3z(fm[1], fm[0], fm[-1], h)


def _inviscid_flux_teno6(Up, velp, pp, cp, grid, d: int, ns: int) -> torch.Tensor:
    """LLF-split TENO6 flux: face f (between cells f-1 and f) takes f+ from cells
    f-3 .. f+2 and f- mirrored (cells f+2 .. f-3); alpha is the maximum of
    |u_n| + c over those six cells."""
    offs = (-3, -2, -1, 0, 1, 2)
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
    return teno6([fp[o] for o in offs]) + teno6([fm[o] for o in reversed(offs)])


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
