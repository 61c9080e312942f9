"""The paper's accuracy problems (Methods, Solver Performance Analysis,
Accuracy) on periodic Cartesian grids, as primitive fields for a single
calorically perfect gas with R/W = 1 (so p = rho T)."""
import math

import numpy as np

from tests.helpers import single_species


def vortex_at(X, Y, t=0.0, L=10.0, beta=5.0, alpha=0.5, r0=0.5, gamma=1.4, u0=1.0, v0=1.0, T0=1.0):
    """Isentropic vortex advected by (u0, v0) at the points (X, Y) (arrays of one
    shape): primitive fields (p, T, u, v, w, Y) of shape (6, 1) + X.shape and rho.
    The exact solution at time t is the initial field translated by (u0 t, v0 t)
    (periodic images ignored).

    The temperature deficit carries the factor r0^2 that radial momentum balance
    requires, (gamma-1) beta^2 r0^2 / (16 alpha gamma pi^2); the printed form
    omits it, which is exact only for r0 = 1."""
    Xc = (X - u0 * t + L / 2) % L - L / 2
    Yc = (Y - v0 * t + L / 2) % L - L / 2
    ex = np.exp(alpha * (1.0 - (Xc ** 2 + Yc ** 2) / r0 ** 2))
    u = beta / (2 * math.pi) * ex * Yc + u0
    v = -beta / (2 * math.pi) * ex * Xc + v0
    T = -(gamma - 1.0) * beta ** 2 * r0 ** 2 / (16.0 * alpha * gamma * math.pi ** 2) * ex ** 2 + T0
    rho = T ** (1.0 / (gamma - 1.0))
    p = rho ** gamma
    sh = (1,) + X.shape
    prim = np.stack([p.reshape(sh), (p / rho).reshape(sh), u.reshape(sh), v.reshape(sh),
                     np.zeros(sh), np.ones(sh)])
    return prim, rho


def vortex_prim(N, t=0.0, L=10.0, **kw):
    """The vortex on the N x N Cartesian grid of [-L/2, L/2]^2 (cell centres)."""
    dx = L / N
    x = -L / 2 + (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")            # [ny, nx]
    prim, rho = vortex_at(X, Y, t, L, **kw)
    return prim, rho, dx


def tgv_prim(N, L=2 * math.pi, gamma=1.4, mu=1.0, rho0=1.0, u0=1.0):
    """2-D Taylor-Green vortex with Re0 = rho0 u0 L / mu = L and
    Ma0 = u0 / sqrt(gamma p0 / rho0) = 1e-2 / sqrt(gamma)."""
    p0 = rho0 * u0 ** 2 / (gamma * (1e-2 / math.sqrt(gamma)) ** 2)
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    k = 2 * math.pi / L
    u = u0 * np.sin(k * X) * np.cos(k * Y)
    v = -u0 * np.cos(k * X) * np.sin(k * Y)
    p = p0 - rho0 * u0 ** 2 / 4.0 * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    rho = np.full_like(p, rho0)
    sh = (1, N, N)
    prim = np.stack([p.reshape(sh), (p / rho).reshape(sh), u.reshape(sh), v.reshape(sh),
                     np.zeros(sh), np.ones(sh)])
    return prim, dx, p0


def tgv_exact_u(N, t, L=2 * math.pi, mu=1.0, rho0=1.0, u0=1.0):
    dx = L / N
    x = (np.arange(N) + 0.5) * dx
    X, Y = np.meshgrid(x, x, indexing="xy")
    k = 2 * math.pi / L
    return u0 * np.sin(k * X) * np.cos(k * Y) * math.exp(-2.0 * mu / rho0 * k * k * t)


def gas(mu=0.0):
    return single_species(gamma=1.4, W=8.314462618, mu=mu, mu_exp=0.0)
