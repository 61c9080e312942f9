"""Curvilinear (mapped) grids (Methods, Numerical method: the mapped equations;
Solver Performance Analysis, Accuracy: the skewed-grid tests) through the C ABI
against the FP64 oracle on the same seeded inputs: the FP64 RHS within 1e-12 per
conserved variable (of its group's scale; momentum at least of the pressure-force
scale p / h, see _err_mapped) with WENO3-Z and TENO6 on the paper's skewed grid,
curved periodic and non-periodic 3-D grids and a uniform grid given by its nodes;
FP64 RK steps at the time-step rule likewise; the mixed path within 1e-4 of those
scales per RHS and 1e-5 after a run of steps; a uniform flow stays uniform; the
skewed-grid vortex converges at third order on the GPU; characteristic (NSCBC)
ends on curved grids match the oracle likewise; the entry points that do not support
mapped grids reject them."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2202_02319_b300 import synth
from tests import cases_accuracy as ca
from tests.gpu_common import gpu_setup, laser_tuple, oracle_setup, rel_inf, state_rel_l2
from tests.helpers import random_prim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _perturbed(nx, ny, nz, h, seed, amp=0.15):
    g = np.random.default_rng(seed)
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = np.stack([i * h, j * h, k * h]).astype(np.float64)
    for c in range(3):
        ph = g.uniform(0, 2 * np.pi, 3)
        X[c] += amp * h * np.sin(0.7 * i + ph[0]) * np.cos(0.9 * j + ph[1]) * np.sin(0.8 * k + ph[2])
    return X


def _case(name, shape, nodes, bc, seed, laser=True):
    m = synth.mechanism_9sp(seed)
    nz, ny, nx = shape
    grid = synth.Grid(nx, ny, nz, 1e-4, 1e-4, 1e-4, bc)
    prim = random_prim(m, shape, seed, smooth=True)
    las = synth.Laser()
    if laser:
        C = nodes.reshape(3, -1).mean(1)
        las = synth.Laser(E=1e-5, x0=float(C[0]), y0=float(C[1]), z0=float(C[2]), sigma_r=2e-4, t0=0.0, sigma_t=1e-8)
    return synth.Case(name, m, grid, prim, las, nodes=nodes)


def _cases():
    N = 24
    skew = synth.skewed_nodes(N, L=N * 1e-4)
    return [_case("skewed_24x24", (1, N, N), skew, (0, 0, 0), 1),
            _case("wavy_10x9x8", (8, 9, 10), synth.wavy_nodes(10, 9, 8, 1e-4), (0, 0, 0), 2),
            _case("perturbed_12x7x6", (6, 7, 12), _perturbed(12, 7, 6, 1e-4, 3), (0, 1, 1), 3),
            _case("row_300x3x2", (2, 3, 300), synth.wavy_nodes(300, 3, 2, 1e-4, 0.1), (0, 0, 1), 4, laser=False)]


CASES = _cases()


def _oracle_rhs(case, flags=None):
    mt, g, Uo, To = oracle_setup(case)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, laser_tuple(case), flags)
    return ro


def _err_mapped(out, ro, case):
    """Per-variable max error over the largest value of the variable's group
    (species, momentum, energy); momentum at least over the pressure-force scale
    p_max / h.  On a curved grid the momentum RHS is the difference of face pressure
    forces p S_k of size p |S| / V that do not cancel face by face, so rounding at
    that scale is the attainable agreement: the oracle itself moves by up to 2e-11
    of the momentum RHS (TENO6 on the skewed grid) when its input is perturbed by one
    ulp."""
    ns = case.mech.n_species
    a = out.reshape(out.shape[0], -1).double().cpu()
    b = ro.reshape(ro.shape[0], -1).double().cpu()
    num = (a - b).abs().amax(1)
    m = b.abs().amax(1)
    p_max = float(np.max(case.prim[0]))
    scale = torch.cat([m[:ns].max().repeat(ns), torch.clamp(m[ns:ns + 3].max(), min=p_max / case.grid.dx).repeat(3),
                       m[ns + 3:]])
    return (num / scale).numpy()


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_mapped_rhs_parity_fp64(case, teno):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6 if teno else 0)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    ro = _oracle_rhs(case, {"scheme": "teno6"} if teno else None)
    err = _err_mapped(out, ro, case)
    assert err.max() < TOL64, err


@pytest.mark.parametrize("flags", [1, 2])
def test_mapped_rhs_parity_term_switches(flags):
    """Viscous part alone (inviscid off) and inviscid part alone on the curved grid."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=flags)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    ro = _oracle_rhs(case, {"inviscid": not (flags & 1), "viscous": not (flags & 2)})
    assert _err_mapped(out, ro, case).max() < TOL64


def test_uniform_nodes_match_the_cartesian_gpu_path():
    """A uniform grid given by its nodes gives the Cartesian GPU RHS (FP64)."""
    nv = _nv()
    m = synth.mechanism_9sp(5)
    nz, ny, nx = 7, 8, 9
    prim = random_prim(m, (nz, ny, nx), 5, smooth=True)
    grid = synth.Grid(nx, ny, nz, 1.1e-4, 0.9e-4, 1.3e-4, (0, 1, 0))
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    nodes = np.stack([i * 1.1e-4, j * 0.9e-4, k * 1.3e-4]).astype(np.float64)
    las = synth.Laser(E=2e-3, x0=4.2e-4, y0=3.1e-4, z0=4.4e-4, sigma_r=2e-4, t0=0.0, sigma_t=1e-8)
    cart = synth.Case("cart", m, grid, prim, las)
    mapd = synth.Case("mapped", m, grid, prim, las, nodes=nodes)
    outs = []
    for c in (cart, mapd):
        mech, ctx, U, T = gpu_setup(c)
        out = torch.empty_like(U)
        nv.rhs(ctx, U, T, 0.0, las.as_tuple(), out)
        nv.check(ctx)
        outs.append(out)
    assert _err_mapped(outs[1], outs[0], mapd).max() < TOL64


@pytest.mark.parametrize("case", [CASES[0], CASES[1]], ids=[CASES[0].name, CASES[1].name])
def test_mapped_rhs_parity_mixed(case):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, laser_tuple(case), out)
    nv.check(ctx)
    err = _err_mapped(out, _oracle_rhs(case), case)
    assert err.max() < 1e-4, err


def test_mapped_rk_step_parity_fp64():
    """Three FP64 steps at the CFL rule on the curved periodic grid, the time step
    chosen by each side."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    las = laser_tuple(case)
    to = 0.0
    for _ in range(3):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, las, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, las, 0.5)
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf(U, Uo.reshape(U.shape)).max() < TOL64


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
def test_mapped_mixed_precision_state_error(teno):
    """Mixed path against the FP64 oracle after 20 steps of 2 ns on the skewed grid,
    laser on: group-scaled relative L2 within 1e-5."""
    nv = _nv()
    case = CASES[0]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED, flags=nv.RF_TENO6 if teno else 0)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    las = laser_tuple(case)
    fl = {"scheme": "teno6"} if teno else None
    dt = 2e-9
    for k in range(20):
        nv.rk_step(ctx, U, T, t, dt, 0.5, las, None)
        Uo, To, _ = oracle.rk.rk_step(mt, g, Uo, To, k * dt, dt, las, 0.5, fl)
    nv.check(ctx)
    err = state_rel_l2(U, Uo, case.mech.n_species)
    assert err.max() < 1e-5, err


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_uniform_flow_stays_uniform(precision):
    """A uniform flow on the skewed and the curved grids: |dU/dt| below 1e-12 (FP64)
    or 1e-5 (mixed) of the scale rho c / h of each group."""
    nv = _nv()
    for base in CASES[:2]:
        m = base.mech
        prim = np.zeros_like(base.prim)
        prim[0], prim[1], prim[2], prim[3], prim[4] = 101325.0, 600.0, 80.0, -40.0, 25.0
        prim[5:] = np.asarray(synth._air(m))[:, None, None, None]
        case = synth.Case("uniform", m, base.grid, prim, synth.Laser(), nodes=base.nodes)
        mech, ctx, U, T = gpu_setup(case, precision=precision)
        out = torch.empty_like(U)
        nv.rhs(ctx, U, T, 0.0, None, out)
        nv.check(ctx)
        ns = m.n_species
        rho = float(U[:ns].sum(0).max())
        c = 600.0
        scale = torch.tensor([rho] * ns + [rho * c] * 3 + [float(U[-1].max())], dtype=torch.float64,
                             device="cuda")[:, None] * c / 1e-4
        bar = 1e-12 if precision == 0 else 1e-5
        assert float((out.abs() / scale).max()) < bar


def _gpu_skewed_vortex_error(N, L=10.0):
    nv = _nv()
    nodes = synth.skewed_nodes(N, L)
    C = nodes.reshape(3, 2, N + 1, N + 1)
    Xc = 0.25 * (C[0, 0, :-1, :-1] + C[0, 0, 1:, :-1] + C[0, 0, :-1, 1:] + C[0, 0, 1:, 1:])
    Yc = 0.25 * (C[1, 0, :-1, :-1] + C[1, 0, 1:, :-1] + C[1, 0, :-1, 1:] + C[1, 0, 1:, 1:])
    prim, _ = ca.vortex_at(Xc, Yc, 0.0, L)
    grid = synth.Grid(N, N, 1, L / N, L / N, L / N, (0, 0, 0))
    case = synth.Case("vortex", ca.gas(), grid, prim, synth.Laser(), nodes=nodes)
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_NO_VISCOUS | nv.RF_NO_CHEMISTRY | nv.RF_NO_LASER)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    for _ in range(50):
        nv.rk_step(ctx, U, T, t, 1e-3, 0.5, None, None)
    nv.check(ctx)
    _, rex = ca.vortex_at(Xc, Yc, 0.05, L)
    return float(np.abs(U[0].reshape(N, N).cpu().numpy() - rex).mean())


def test_skewed_grid_vortex_converges_at_third_order_on_the_gpu():
    """Accuracy problem 1 on the paper's skewed grid (t = 0.05), FP64 WENO3-Z on the
    GPU: the L1 error of rho falls at third order between N = 64 and 128."""
    e = [_gpu_skewed_vortex_error(N) for N in (32, 64, 128)]
    assert math.log2(e[1] / e[2]) > 2.6, e


def test_mapped_diagnostics_integrate_with_cell_volumes():
    nv = _nv()
    case = CASES[2]
    mech, ctx, U, T = gpu_setup(case)
    d = nv.diagnostics(ctx, U, T)
    mt, g, Uo, To = oracle_setup(case)
    V = oracle.mapped.geometry(g)["V"]
    tot = (Uo * V[None]).reshape(Uo.shape[0], -1).sum(1).numpy()
    assert np.allclose(d["total"], tot, rtol=1e-12, atol=0.0)


def test_mapped_is_rejected_where_unsupported():
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    ens = nv.ensemble_create([ctx], [U], [T], [case.laser.as_tuple()], t)
    with pytest.raises(RuntimeError, match="Cartesian members"):
        nv.run_ensemble(ens, 1, nv.ENS_GRAPH, 0.5)
    code, st = nv.run_ensemble(ens, 1, nv.ENS_LOOP, 0.5)
    assert code == 0 and float(t[0]) > 0.0
    del ens
    lam = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="RF_MAPPED"):
        nv.adjoint_rhs(ctx, U, T, 0.0, None, lam, 0.0, lam.clone(), grads)
    fresh = nv.create_ctx(mech, case.grid, nv.RF_FP64, nv.RF_MAPPED)
    out = torch.empty_like(U)
    with pytest.raises(RuntimeError, match="rf_set_nodes"):
        nv.rhs(fresh, U, T, 0.0, None, out)
    mirrored = np.ascontiguousarray(case.nodes.copy())
    mirrored[0] = -mirrored[0]                 # left-handed: every volume negative
    with pytest.raises(RuntimeError, match="non-positive"):
        nv.set_nodes(fresh, torch.as_tensor(mirrored, dtype=torch.float64).cuda())
    with pytest.raises(RuntimeError, match="RF_MAPPED"):
        nv.set_nodes(nv.create_ctx(mech, case.grid, nv.RF_FP64), torch.as_tensor(case.nodes).cuda())


def _mapped_nscbc_cases():
    """Characteristic ends on curved grids: the paper's skewed grid with an inflow
    target on the low x end and an outflow on the high end; a curved 3-D grid with
    outflows on x and an inflow / outflow pair on y."""
    N = 20
    skew = _case("skewed_nscbc_20x20", (1, N, N), synth.skewed_nodes(N, L=N * 1e-4), (2, 0, 0), 6, laser=False)
    g = np.random.default_rng(6)
    ns = skew.mech.n_species
    tg = np.empty((4 + ns, N))
    tg[0] = 40.0 + 10.0 * g.standard_normal(N)
    tg[1] = 5.0 * g.standard_normal(N)
    tg[2] = 0.0
    tg[3] = 900.0
    Y = g.dirichlet(np.ones(ns), size=N).T
    tg[4:] = Y
    skew.nscbc = {(0, 0): dict(p_inf=101325.0, eta_u=0.8, eta_T=1.2, eta_t=0.6, eta_Y=0.9, target=tg),
                  (0, 1): dict(p_inf=100000.0, sigma=0.3, target=None)}
    wavy = _case("wavy_nscbc_10x9x8", (8, 9, 10), synth.wavy_nodes(10, 9, 8, 1e-4), (2, 2, 0), 7, laser=False)
    tgy = np.empty((4 + ns, 10 * 8))
    tgy[0], tgy[1], tgy[2], tgy[3] = 10.0, 30.0, -5.0, 800.0
    tgy[4:] = (np.ones(ns) / ns)[:, None]
    wavy.nscbc = {(0, 0): dict(p_inf=101325.0, sigma=0.25, target=None),
                  (0, 1): dict(p_inf=101325.0, sigma=0.5, target=None),
                  (1, 0): dict(p_inf=101325.0, eta_u=1.5, eta_T=0.5, eta_t=1.0, eta_Y=0.7, length=2e-3, target=tgy),
                  (1, 1): dict(p_inf=99000.0, sigma=0.1, target=None)}
    return [skew, wavy]


NSCBC_CASES = _mapped_nscbc_cases()


def _oracle_rhs_nscbc(case, flags=None):
    from tests.gpu_common import nscbc_oracle
    return _oracle_rhs(case, dict(flags or {}, nscbc=nscbc_oracle(case)))


@pytest.mark.parametrize("teno", [False, True], ids=["weno3z", "teno6"])
@pytest.mark.parametrize("case", NSCBC_CASES, ids=[c.name for c in NSCBC_CASES])
def test_mapped_nscbc_rhs_parity_fp64(case, teno):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_TENO6 if teno else 0)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, None, out)
    nv.check(ctx)
    err = _err_mapped(out, _oracle_rhs_nscbc(case, {"scheme": "teno6"} if teno else None), case)
    assert err.max() < TOL64, err


@pytest.mark.parametrize("case", NSCBC_CASES, ids=[c.name for c in NSCBC_CASES])
def test_mapped_nscbc_rhs_parity_mixed(case):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, None, out)
    nv.check(ctx)
    err = _err_mapped(out, _oracle_rhs_nscbc(case), case)
    assert err.max() < 1e-4, err


def test_mapped_nscbc_rk_step_parity_fp64():
    """Three FP64 steps at the CFL rule with characteristic ends on the skewed grid."""
    from tests.gpu_common import nscbc_oracle
    nv = _nv()
    case = NSCBC_CASES[0]
    mech, ctx, U, T = gpu_setup(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    fl = {"nscbc": nscbc_oracle(case)}
    to = 0.0
    for _ in range(3):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, None, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, None, 0.5, fl)
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf(U, Uo.reshape(U.shape)).max() < TOL64
