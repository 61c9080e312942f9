"""Pins of the oracle's mapped (curvilinear) form (Methods, Numerical method: the
mapped equations; Solver Performance Analysis, Accuracy: the skewed-grid
convergence tests), each against something outside the mapped code: the
Cartesian oracle (a uniform grid given by its nodes, and a rotated grid carrying
one-dimensional data), the exact invariants of a conservative, freestream-
preserving discretisation, and the paper's skewed-grid vortex."""
import math

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth
from oracle import mapped, rhs, rk
from oracle.mech import GridT
from tests import cases_accuracy as ca
from tests.helpers import mech_t, random_prim, tensor

NOSRC = {"chemistry": False, "laser": False}


def cartesian_nodes(nx, ny, nz, dx, dy, dz, origin=(0.0, 0.0, 0.0)):
    i = torch.arange(nx + 1, dtype=torch.float64) * dx + origin[0]
    j = torch.arange(ny + 1, dtype=torch.float64) * dy + origin[1]
    k = torch.arange(nz + 1, dtype=torch.float64) * dz + origin[2]
    Z, Y, X = torch.meshgrid(k, j, i, indexing="ij")
    return torch.stack([X, Y, Z])


def skewed_nodes(N, L=10.0, beta=0.2, dz=None):
    """The paper's skewed grid: the uniform N x N nodes (xi, eta) of [-L/2, L/2]^2
    placed at x = xi (1 + beta sin(2 pi eta / L)), y = eta (1 + beta sin(2 pi xi / L));
    one cell deep (z nodes 0 and dz)."""
    h = L / N
    s = -L / 2 + torch.arange(N + 1, dtype=torch.float64) * h
    E, Xi = torch.meshgrid(s, s, indexing="ij")               # [ny+1, nx+1]
    x = Xi * (1.0 + beta * torch.sin(2 * math.pi * E / L))
    y = E * (1.0 + beta * torch.sin(2 * math.pi * Xi / L))
    dz = h if dz is None else dz
    X = torch.stack([x, x])
    Y = torch.stack([y, y])
    Z = torch.stack([torch.zeros_like(x), torch.full_like(x, dz)])
    return torch.stack([X, Y, Z])


def _state(m, shape, seed):
    mt = mech_t(m)
    prim = tensor(random_prim(m, shape, seed, smooth=True))
    U, T = rhs.init_state(mt, prim)
    return mt, U, T


def _rel(a, b):
    num = (a - b).reshape(a.shape[0], -1).abs().amax(1)
    den = b.reshape(b.shape[0], -1).abs().amax(1)
    return (num / torch.where(den > 0, den, torch.ones_like(den))).max().item()


@pytest.mark.parametrize("scheme", ["weno3z", "teno6"])
def test_uniform_cartesian_nodes_reproduce_the_cartesian_rhs(scheme):
    """A uniform grid given by its nodes runs the mapped form to the Cartesian RHS
    (all terms: inviscid, viscous, chemistry, laser) and the same time step."""
    m = synth.mechanism_4sp(0)
    nz, ny, nx = 5, 6, 7
    dx, dy, dz = 1.1e-4, 0.9e-4, 1.3e-4
    mt, U, T = _state(m, (nz, ny, nx), 2)
    bc = (0, 1, 0)
    gc = GridT(nx, ny, nz, dx, dy, dz, bc)
    gm = mapped.MappedGridT(nx, ny, nz, cartesian_nodes(nx, ny, nz, dx, dy, dz), bc)
    las = (2e-3, 3.3 * dx, 2.6 * dy, 2.2 * dz, 2.0 * dx, 0.0, 1e-8)
    fl = {"scheme": scheme}
    rc, _ = rhs.rhs(mt, gc, U, T, 0.0, las, fl)
    rm, _ = rhs.rhs(mt, gm, U, T, 0.0, las, fl)
    assert _rel(rm, rc) < 1e-12
    dtc = rk.time_step(mt, gc, U, T, 0.0, None, 0.5)
    dtm = rk.time_step(mt, gm, U, T, 0.0, None, 0.5)
    assert dtm == pytest.approx(dtc, rel=1e-13)


def _uniform_state(mt, shape, u=(80.0, -40.0, 25.0), p=101325.0, T=600.0, Y=(0.1, 0.2, 0.3, 0.4)):
    prim = torch.empty((9,) + shape, dtype=torch.float64)
    prim[0], prim[1] = p, T
    for k in range(3):
        prim[2 + k] = u[k]
    prim[5:] = torch.tensor(Y, dtype=torch.float64)[:, None, None, None]
    return rhs.init_state(mt, prim)


def _perturbed_nodes(nx, ny, nz, h, seed, amp=0.15):
    """Uniform nodes moved by a smooth random displacement of amplitude amp h."""
    X = cartesian_nodes(nx, ny, nz, h, h, h)
    g = np.random.default_rng(seed)
    k = torch.arange(nz + 1, dtype=torch.float64)[:, None, None]
    j = torch.arange(ny + 1, dtype=torch.float64)[None, :, None]
    i = torch.arange(nx + 1, dtype=torch.float64)[None, None, :]
    for c in range(3):
        ph = g.uniform(0, 2 * math.pi, 3)
        X[c] = X[c] + amp * h * (torch.sin(0.7 * i + ph[0]) * torch.cos(0.9 * j + ph[1]) * torch.sin(0.8 * k + ph[2]))
    return X


@pytest.mark.parametrize("scheme", ["weno3z", "teno6"])
def test_uniform_flow_stays_uniform_on_skewed_grids(scheme):
    """Freestream preservation: a uniform flow (viscous terms on) has a zero RHS
    to rounding on the paper's skewed grid (periodic seam included) and on a
    randomly perturbed 3-D grid."""
    mt = mech_t(synth.mechanism_4sp(0))
    N = 16
    grids = [mapped.MappedGridT(N, N, 1, skewed_nodes(N, L=N * 1e-4), (0, 0, 0)),
             mapped.MappedGridT(7, 6, 5, _perturbed_nodes(7, 6, 5, 1e-4, 3), (0, 1, 1))]
    for g in grids:
        U, T = _uniform_state(mt, (g.nz, g.ny, g.nx))
        R, _ = rhs.rhs(mt, g, U, T, 0.0, None, dict(NOSRC, scheme=scheme))
        st = rhs.primitives(mt, U, T)
        rho, c = float(st["rho"].max()), float(st["c"].max())
        scale = torch.tensor([rho] * 4 + [rho * c] * 3 + [float(U[-1].max())],
                             dtype=torch.float64)[:, None, None, None] * c / 1e-4
        assert float((R.abs() / scale).max()) < 1e-12


def test_periodic_mapped_grid_conserves_mass_momentum_energy():
    """On a translation-periodic curved grid the sum over cells of V dU/dt vanishes
    (no chemistry, no laser): every face flux leaves one cell and enters the next."""
    m = synth.mechanism_4sp(0)
    nz, ny, nx = 4, 6, 8
    h = 1e-4
    mt, U, T = _state(m, (nz, ny, nx), 5)
    X = cartesian_nodes(nx, ny, nz, h, h, h)
    k = torch.arange(nz + 1, dtype=torch.float64)[:, None, None]
    j = torch.arange(ny + 1, dtype=torch.float64)[None, :, None]
    i = torch.arange(nx + 1, dtype=torch.float64)[None, None, :]
    X[0] = X[0] + 0.2 * h * torch.sin(2 * math.pi * j / ny) * torch.cos(2 * math.pi * k / nz)
    X[1] = X[1] + 0.15 * h * torch.sin(2 * math.pi * i / nx + 0.3) + 0.1 * h * torch.cos(2 * math.pi * k / nz)
    X[2] = X[2] + 0.1 * h * torch.sin(2 * math.pi * (i / nx + j / ny))
    g = mapped.MappedGridT(nx, ny, nz, X, (0, 0, 0))
    R, _ = rhs.rhs(mt, g, U, T, 0.0, None, NOSRC)
    V = mapped.geometry(g)["V"]
    tot = (R * V[None]).reshape(R.shape[0], -1).sum(1)
    mag = (R * V[None]).reshape(R.shape[0], -1).abs().sum(1)
    assert float((tot.abs() / mag).max()) < 1e-12


@pytest.mark.parametrize("scheme", ["weno3z", "teno6"])
def test_rotated_grid_carries_one_dimensional_data_like_the_cartesian_grid(scheme):
    """A uniform grid rotated by 30 degrees with data varying along its first axis
    only and the velocity along that axis: the RHS is the one-dimensional
    Cartesian RHS with the momentum rotated (component-wise reconstruction of two
    proportional momentum components gives proportional values)."""
    m = synth.mechanism_4sp(0)
    nx, ny, h = 24, 3, 1e-4
    mt = mech_t(m)
    prim1 = tensor(random_prim(m, (1, 1, nx), 7, smooth=True))
    prim1[3] = 0.0
    prim1[4] = 0.0
    th = math.radians(30.0)
    cs, sn = math.cos(th), math.sin(th)
    X = cartesian_nodes(nx, ny, 1, h, h, h)
    Xr = X.clone()
    Xr[0] = cs * X[0] - sn * X[1]
    Xr[1] = sn * X[0] + cs * X[1]
    g2 = mapped.MappedGridT(nx, ny, 1, Xr, (0, 0, 0))
    prim2 = prim1.expand(prim1.shape[0], 1, ny, nx).clone()
    prim2[2] = cs * prim1[2]
    prim2[3] = sn * prim1[2]
    U2, T2 = rhs.init_state(mt, prim2)
    U1, T1 = rhs.init_state(mt, prim1)
    fl = dict(NOSRC, scheme=scheme)
    R2, _ = rhs.rhs(mt, g2, U2, T2, 0.0, None, fl)
    R1, _ = rhs.rhs(mt, GridT(nx, 1, 1, h, h, h, (0, 0, 0)), U1, T1, 0.0, None, fl)
    want = R1.expand(R1.shape[0], 1, ny, nx).clone()
    ns = 4
    want[ns] = cs * R1[ns]
    want[ns + 1] = sn * R1[ns]
    scale = R1.reshape(R1.shape[0], -1).abs().amax(1)
    scale[ns + 1] = scale[ns]
    scale[ns + 2] = scale[ns]
    err = (R2 - want).reshape(R2.shape[0], -1).abs().amax(1) / scale
    assert float(err.max()) < 1e-11


def _skewed_vortex_error(N, scheme="weno3z", L=10.0):
    mt = mech_t(ca.gas())
    g = mapped.MappedGridT(N, N, 1, skewed_nodes(N, L), (0, 0, 0))
    C = mapped.geometry(g)["C"]
    X, Y = C[0, 0].numpy(), C[1, 0].numpy()
    prim, _ = ca.vortex_at(X, Y, 0.0, L)
    U, T = rhs.init_state(mt, tensor(prim))
    fl = {"viscous": False, "chemistry": False, "laser": False, "scheme": scheme}
    t, dt = 0.0, 1e-3
    for _ in range(50):
        U, T, _ = rk.rk_step(mt, g, U, T, t, dt, None, flags=fl)
        t += dt
    _, rex = ca.vortex_at(X, Y, t, L)
    return float(np.abs(U[0, 0].numpy() - rex).mean())


def test_skewed_grid_vortex_converges_at_third_order():
    """Accuracy problem 1 on the paper's skewed grid (beta = 0.2, L = 10, t = 0.05):
    the L1 error of rho with WENO3-Z falls at third order between N = 64 and 128,
    the rate the paper reports on these grids."""
    e = [_skewed_vortex_error(N) for N in (32, 64, 128)]
    assert math.log2(e[1] / e[2]) > 2.6, e
