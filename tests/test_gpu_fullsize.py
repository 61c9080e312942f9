"""Parity at the benchmark's full size (256^3 jet in a box, 9 species, laser on)
in the launch configuration bench.py times.  The oracle cannot evaluate the
whole grid, so it evaluates sampled cells one by one: the RHS of a cell depends
only on cells within two of it (one RK step: within six), so the oracle runs on
a periodic patch around the sample cut from the same seeded input, and the
patch's centre is exact."""
import numpy as np
import pytest
import torch

import oracle
from oracle.mech import GridT, from_synth, grid_from_synth
from paper_2202_02319_b300 import synth

pytestmark = pytest.mark.gpu

N = 256


@pytest.fixture(scope="module")
def jet():
    case = synth.case_jet(0, N, device="cuda")
    return case


def _samples(case, k, seed):
    g = np.random.default_rng(seed)
    pts = [tuple(int(v) for v in g.integers(0, N, 3)) for _ in range(k)]
    dx = case.grid.dx
    lc = (int(case.laser.x0 / dx), int(case.laser.y0 / dx), int(case.laser.z0 / dx))
    pts += [lc, (lc[0] + 2, lc[1] - 1, lc[2] + 1), (N // 2, N // 2 + 16, N // 2), (N // 2, N // 2, N // 2 - 17)]
    return pts


def _patch(case, c, r):
    """Primitive fields of the (2r+1)^3 periodic patch centred on cell c = (i, j, k)."""
    i, j, k = c
    ii = torch.arange(i - r, i + r + 1, device=case.prim.device) % N
    jj = torch.arange(j - r, j + r + 1, device=case.prim.device) % N
    kk = torch.arange(k - r, k + r + 1, device=case.prim.device) % N
    p = case.prim.index_select(1, kk).index_select(2, jj).index_select(3, ii)
    return p.double().cpu().contiguous()


def _patch_laser(case, c, r):
    las = list(case.laser.as_tuple())
    dx = case.grid.dx
    las[1] -= (c[0] - r) * dx
    las[2] -= (c[1] - r) * dx
    las[3] -= (c[2] - r) * dx
    return tuple(las)


def _gpu_state(case, precision, flags=0):
    from paper_2202_02319_b300 import native as nv
    ns = case.mech.n_species
    n = case.grid.ncells
    mech = nv.init_mechanism(case.mech)
    ctx = nv.create_ctx(mech, case.grid, precision, flags)
    U = torch.empty((ns + 4, n), dtype=torch.float64, device="cuda")
    T = torch.empty(n, dtype=torch.float64, device="cuda")
    nv.init_state(ctx, case.prim.reshape(5 + ns, n), U, T)
    nv.check(ctx)
    return mech, ctx, U, T


def _group_scale(v, ns):
    """Per-variable comparison scale: the max over its group (species block,
    momentum block, energy)."""
    sc = torch.empty_like(v)
    sc[:ns] = v[:ns].max()
    sc[ns:ns + 3] = v[ns:ns + 3].max()
    sc[ns + 3] = v[ns + 3]
    return sc


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-4)], ids=["fp64", "mixed"])
def test_fullsize_rhs_sampled(jet, precision, tol):
    from paper_2202_02319_b300 import native as nv
    case = jet
    ns = case.mech.n_species
    mech, ctx, U, T = _gpu_state(case, precision)
    out = torch.empty_like(U)
    t = case.laser.t0
    nv.rhs(ctx, U, T, t, case.laser.as_tuple(), out)
    nv.check(ctx)
    assert bool(torch.isfinite(out).all())
    mt = from_synth(case.mech)
    g = GridT(5, 5, 5, case.grid.dx, case.grid.dy, case.grid.dz)
    gpu, orc = [], []
    for c in _samples(case, 24, 1):
        Up, Tp = oracle.rhs.init_state(mt, _patch(case, c, 2))
        ro, _ = oracle.rhs.rhs(mt, g, Up, Tp, t, _patch_laser(case, c, 2))
        orc.append(ro[:, 2, 2, 2])
        gpu.append(out[:, (c[2] * N + c[1]) * N + c[0]].cpu())
    gpu, orc = torch.stack(gpu, 1), torch.stack(orc, 1)
    scale = _group_scale(orc.abs().amax(1), ns) if precision else orc.abs().amax(1)
    diff = (gpu - orc).abs().amax(1)
    err = torch.where(scale > 0, diff / torch.where(scale > 0, scale, torch.ones_like(scale)), diff).numpy()
    assert err.max() < tol, err


SCHEMES = [("teno6", 16, {"scheme": "teno6"}, 3), ("charwise_weno3z", 64, {"splitting": "characteristic"}, 2),
           ("charwise_teno6", 80, {"scheme": "teno6", "splitting": "characteristic"}, 3)]


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("name,flags,ofl,r", SCHEMES, ids=[x[0] for x in SCHEMES])
def test_fullsize_rhs_sampled_other_schemes(jet, name, flags, ofl, r, precision):
    """TENO6 and characteristic-wise splitting (WENO3-Z, TENO6) at 256^3 in FP64, in the
    configuration the bench's legs time, on sampled cells (patch radius r: the scheme's
    halo).  TENO6: 1e-12 per variable.  Characteristic-wise: 1e-12 of the group's
    largest sampled value, or twice the oracle's own movement at the sample under a
    one-ulp perturbation of the patch state where that is larger (the projection
    cancels terms of the size of the species energies, so its rounding does not scale
    with the RHS).  Mixed precision: 1e-4 of the group's largest sampled value, the
    mixed RHS bar of the WENO3-Z test above."""
    from paper_2202_02319_b300 import native as nv
    case = jet
    ns = case.mech.n_species
    mech, ctx, U, T = _gpu_state(case, precision, flags)
    out = torch.empty_like(U)
    t = case.laser.t0
    nv.rhs(ctx, U, T, t, case.laser.as_tuple(), out)
    nv.check(ctx)
    assert bool(torch.isfinite(out).all())
    mt = from_synth(case.mech)
    w = 2 * r + 1
    g = GridT(w, w, w, case.grid.dx, case.grid.dy, case.grid.dz)
    gen = torch.Generator().manual_seed(5)
    gpu, orc, noise = [], [], []
    for c in _samples(case, 16, 2):
        Up, Tp = oracle.rhs.init_state(mt, _patch(case, c, r))
        las = _patch_laser(case, c, r)
        ro, _ = oracle.rhs.rhs(mt, g, Up, Tp, t, las, ofl)
        orc.append(ro[:, r, r, r])
        gpu.append(out[:, (c[2] * N + c[1]) * N + c[0]].cpu())
        if "splitting" in ofl and precision == 0:
            xi = torch.randint(0, 2, Up.shape, generator=gen, dtype=torch.float64) * 2.0 - 1.0
            r1, _ = oracle.rhs.rhs(mt, g, Up * (1.0 + xi * 2.0 ** -52), Tp, t, las, ofl)
            noise.append((r1[:, r, r, r] - ro[:, r, r, r]).abs())
    del out, U, T, ctx
    gpu, orc = torch.stack(gpu, 1), torch.stack(orc, 1)
    diff = (gpu - orc).abs().amax(1)
    tol = 1e-12 if precision == 0 else 1e-4
    if precision:
        scale = _group_scale(orc.abs().amax(1), ns)
    elif noise:
        nz = torch.stack(noise, 1).amax(1)
        scale = torch.maximum(_group_scale(orc.abs().amax(1), ns), 2.0e12 * _group_scale(nz, ns))
    else:
        scale = orc.abs().amax(1)
    err = torch.where(scale > 0, diff / torch.where(scale > 0, scale, torch.ones_like(scale)), diff).numpy()
    print(name, precision, "err", err.max())
    assert err.max() < tol, err


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-6)], ids=["fp64", "mixed"])
def test_fullsize_rk_step_sampled(jet, precision, tol):
    """One SSP-RK3 step at a fixed dt: the state at sampled cells matches the oracle
    stepping a 15^3 periodic patch (radius 7 >= 3 stages x stencil radius 2)."""
    from paper_2202_02319_b300 import native as nv
    case = jet
    ns = case.mech.n_species
    mech, ctx, U, T = _gpu_state(case, precision)
    t = torch.full((1,), case.laser.t0 - 1e-8, dtype=torch.float64, device="cuda")
    dt = 4e-9
    nv.rk_step(ctx, U, T, t, dt, case.cfl, case.laser.as_tuple(), None)
    nv.check(ctx)
    mt = from_synth(case.mech)
    g = GridT(15, 15, 15, case.grid.dx, case.grid.dy, case.grid.dz)
    gpu, orc = [], []
    for c in _samples(case, 3, 2):
        Up, Tp = oracle.rhs.init_state(mt, _patch(case, c, 7))
        Uo, _, _ = oracle.rk.rk_step(mt, g, Up, Tp, case.laser.t0 - 1e-8, dt, _patch_laser(case, c, 7), case.cfl)
        orc.append(Uo[:, 7, 7, 7])
        gpu.append(U[:, (c[2] * N + c[1]) * N + c[0]].cpu())
    gpu, orc = torch.stack(gpu, 1), torch.stack(orc, 1)
    scale = _group_scale(orc.abs().amax(1), ns)
    err = ((gpu - orc).abs().amax(1) / scale).numpy()
    assert err.max() < tol, err


def test_fullsize_time_step_rule(jet):
    """dt from the device reduction equals the oracle's rule over all 256^3 cells
    (the oracle evaluates the pointwise rates slab by slab)."""
    from paper_2202_02319_b300 import native as nv
    case = jet
    mech, ctx, U, T = _gpu_state(case, 0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    nv.rk_step(ctx, U, T, t, 0.0, case.cfl, case.laser.as_tuple(), dt)
    nv.check(ctx)
    mt = from_synth(case.mech)
    ac = dm = ch = 0.0
    slab = 16
    for z0 in range(0, N, slab):
        p = case.prim[:, z0:z0 + slab].double().cpu().contiguous()
        g = GridT(N, N, slab, case.grid.dx, case.grid.dy, case.grid.dz)
        Us, Ts = oracle.rhs.init_state(mt, p)
        a, d, c = oracle.rk.rate_limits(mt, g, Us, Ts)
        ac, dm, ch = max(ac, a), max(dm, d), max(ch, c)
    ref = min(case.cfl / ac, 0.25 * case.grid.dx ** 2 / dm, 0.2 / ch)
    las = case.laser
    lo, hi = las.t0 - 6 * las.sigma_t, las.t0 + 6 * las.sigma_t
    if ref > lo:
        ref = min(ref, max(0.25 * las.sigma_t, lo))
    assert abs(float(dt) - ref) <= 1e-12 * ref
