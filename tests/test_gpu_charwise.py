"""Characteristic-wise flux splitting (RF_CHARWISE; Methods, Numerical method: the
optional reconstruction of characteristic instead of conserved variables) through the
C ABI against the FP64 oracle (oracle.charwise) on the same seeded inputs, with
WENO3-Z and TENO6: the FP64 RHS per conserved variable within the bar below, an FP64
RK step likewise, the mixed path within the 1e-5 state bar after a run of steps; and
the entry points that do not support it reject it (rf_rhs_noalloc's rejection is in
test_zz_no_alloc).

The kernel inverts the face's eigenvectors in closed form, the oracle by an LU solve
(torch.linalg.inv), so the two differ by the rounding of the projection, and that
rounding is set by the terms the projection cancels, not by the result: the species
rows carry Y_s dp / c^2 (dp holds b E and sum_s phi_s rho_s, of the size of b rho e_s
with the species' formation energies) and the energy row |u|^2 - phi_s / b (of the
size of e_s, 1e6..1e7 J/kg), both far above the fluxes they cancel to.  The bar is
therefore the larger of 1e-12 of the group's largest value (species, momentum,
energy: the component-wise scheme's bar) and NOISE_K times the oracle's own
movement (the group's largest) when its input is perturbed by one ulp.  A species
absent from the mixture keeps an exactly zero RHS in the kernel (its eigenvector
entries are exact zeros) and ~1e-20 in the oracle, which the group scale absorbs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2202_02319_b300 import synth
from tests.gpu_common import gpu_setup, laser_tuple, oracle_setup, rel_inf, rel_inf_group, state_rel_l2
from tests.helpers import random_prim

pytestmark = pytest.mark.gpu

TOL64 = 1e-12


def _nv():
    from paper_2202_02319_b300 import native as nv
    return nv


def _random_case(shape, bc, seed, smooth=False):
    m = synth.mechanism_9sp(seed)
    nz, ny, nx = shape
    grid = synth.Grid(nx, ny, nz, 1.1e-4, 0.9e-4, 1.3e-4, bc)
    return synth.Case(f"random{shape}", m, grid, random_prim(m, shape, seed, smooth=smooth))


def _cases():
    jet = synth.case_jet(0, 16)
    jet.laser.t0 = 2e-8
    jet.laser.x0, jet.laser.y0, jet.laser.z0 = 8.3 * jet.grid.dx, 7.6 * jet.grid.dx, 8.1 * jet.grid.dx
    return [synth.case_box32(0), jet, synth.case_mixing_layer(0, 32),
            _random_case((5, 7, 13), (1, 0, 1), 3), _random_case((6, 5, 1), (0, 0, 0), 4),
            _random_case((1, 1, 1), (0, 0, 0), 5), _random_case((2, 3, 300), (0, 1, 0), 6, smooth=True),
            _random_case((4, 5, 257), (0, 0, 1), 8, smooth=True)]


CASES = _cases()
SCHEMES = ["weno3z", "teno6"]


NOISE_K = 2.0


def _oracle_noise(mt, g, Uo, To, las, fl):
    """Per-variable max |RHS(U (1 + 2^-52 xi)) - RHS(U)| of the oracle, xi = +-1 seeded."""
    gen = torch.Generator().manual_seed(7)
    xi = torch.randint(0, 2, Uo.shape, generator=gen, dtype=torch.float64) * 2.0 - 1.0
    r0, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, las, fl)
    r1, _ = oracle.rhs.rhs(mt, g, Uo * (1.0 + xi * 2.0 ** -52), To, 0.0, las, fl)
    return (r1 - r0).reshape(r0.shape[0], -1).abs().amax(1)


def _err_char(out, ro, ns, noise):
    """Per-variable max error over the bar's scale: max(TOL64 x the group's largest
    value, NOISE_K x the group's largest oracle noise) x 1 / TOL64, so that < TOL64
    passes."""
    a = out.reshape(out.shape[0], -1).double().cpu()
    b = ro.reshape(ro.shape[0], -1).double().cpu()
    num = (a - b).abs().amax(1)
    m = b.abs().amax(1)
    groups = [slice(0, ns), slice(ns, ns + 3), slice(ns + 3, ns + 4)]
    scale = torch.empty_like(m)
    for gsl in groups:
        scale[gsl] = torch.maximum(m[gsl].max(), NOISE_K / TOL64 * noise[gsl].max())
    return torch.where(scale > 0, num / torch.where(scale > 0, scale, torch.ones_like(scale)), num).numpy()


def _flags(nv, scheme):
    return nv.RF_CHARWISE | (nv.RF_TENO6 if scheme == "teno6" else 0)


def _ofl(scheme, **kw):
    return dict({"scheme": scheme, "splitting": "characteristic"}, **kw)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("case", CASES, ids=[c.name for c in CASES])
def test_charwise_rhs_parity_fp64(case, scheme):
    nv = _nv()
    mech, ctx, U, T = gpu_setup(case, flags=_flags(nv, scheme))
    out = torch.empty_like(U)
    las = laser_tuple(case)
    nv.rhs(ctx, U, T, 0.0, las, out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, las, _ofl(scheme))
    noise = _oracle_noise(mt, g, Uo, To, las, _ofl(scheme))
    err = _err_char(out, ro, case.mech.n_species, noise)
    d = (out.cpu().reshape(ro.shape[0], -1) - ro.reshape(ro.shape[0], -1)).abs().amax(1)
    print(case.name, scheme, "err", err.max(), "group", rel_inf_group(out, ro, case.mech.n_species).max(),
          "kernel/noise", float((d / noise.clamp_min(1e-300)).max()))
    assert err.max() < TOL64, err


@pytest.mark.parametrize("scheme", SCHEMES)
def test_charwise_inviscid_only(scheme):
    """The inviscid part alone (viscous, chemistry and laser off)."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=_flags(nv, scheme) | nv.RF_NO_VISCOUS | nv.RF_NO_CHEMISTRY | nv.RF_NO_LASER)
    out = torch.empty_like(U)
    nv.rhs(ctx, U, T, 0.0, None, out)
    nv.check(ctx)
    mt, g, Uo, To = oracle_setup(case)
    fl = _ofl(scheme, viscous=False, chemistry=False, laser=False)
    ro, _ = oracle.rhs.rhs(mt, g, Uo, To, 0.0, None, fl)
    err = _err_char(out, ro, case.mech.n_species, _oracle_noise(mt, g, Uo, To, None, fl))
    print("inviscid only", scheme, "err", err.max(), "group", rel_inf_group(out, ro, case.mech.n_species).max())
    assert err.max() < TOL64, err


@pytest.mark.parametrize("scheme", SCHEMES)
def test_charwise_rk_step_parity_fp64(scheme):
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=_flags(nv, scheme))
    las = laser_tuple(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    dt = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    to = 0.0
    for _ in range(2):
        nv.rk_step(ctx, U, T, t, 0.0, 0.5, las, dt)
        nv.check(ctx)
        Uo, To, dto = oracle.rk.rk_step(mt, g, Uo, To, to, 0.0, las, 0.5, _ofl(scheme))
        to += dto
        assert abs(float(dt) - dto) <= 1e-12 * dto
    assert rel_inf_group(U, Uo.reshape(U.shape), case.mech.n_species).max() < 1e-12


@pytest.mark.parametrize("scheme", SCHEMES)
def test_charwise_mixed_precision_state_error(scheme):
    """Mixed path (FP32 bulk, the projection and reconstruction in FP32) against the
    FP64 oracle after 20 steps of the 16^3 jet with the laser on: group-scaled
    relative L2 within 1e-5."""
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, precision=nv.RF_MIXED, flags=_flags(nv, scheme))
    las = laser_tuple(case)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    mt, g, Uo, To = oracle_setup(case)
    dt = 2e-9
    for k in range(20):
        nv.rk_step(ctx, U, T, t, dt, 0.5, las, None)
        Uo, To, _ = oracle.rk.rk_step(mt, g, Uo, To, k * dt, dt, las, 0.5, _ofl(scheme))
    nv.check(ctx)
    err = state_rel_l2(U, Uo, case.mech.n_species)
    print(scheme, "mixed state error", err.max())
    assert err.max() < 1e-5, err


def test_charwise_uniform_state_is_kept():
    """A uniform state gives every face F(U) through the projection and back, so the
    inviscid RHS of a uniform periodic box is zero to rounding, in both precisions."""
    nv = _nv()
    m = synth.mechanism_9sp(2)
    prim = random_prim(m, (4, 5, 6), 2)
    for k in range(prim.shape[0]):
        prim[k] = prim[k].mean()
    case = synth.Case("uniform", m, synth.Grid(6, 5, 4, 1e-4, 1e-4, 1e-4, (0, 0, 0)), prim)
    for prec in (nv.RF_FP64, nv.RF_MIXED):
        for scheme in SCHEMES:
            mech, ctx, U, T = gpu_setup(case, precision=prec, flags=_flags(nv, scheme) | nv.RF_NO_CHEMISTRY | nv.RF_NO_LASER)
            out = torch.empty_like(U)
            nv.rhs(ctx, U, T, 0.0, None, out)
            nv.check(ctx)
            scale = U.abs().amax(1) / 1e-4 * 1e3          # |U| / h times a speed
            tol = 1e-12 if prec == nv.RF_FP64 else 1e-5
            assert float((out.abs().amax(1) / scale).max()) < tol, (prec, scheme)


def test_charwise_is_rejected_where_unsupported():
    nv = _nv()
    case = CASES[1]
    mech, ctx, U, T = gpu_setup(case, flags=nv.RF_CHARWISE)
    t = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="RF_CHARWISE"):
        nv.ensemble_create([ctx], [U], [T], [case.laser.as_tuple()], t)
    lam = torch.zeros_like(U)
    grads = torch.zeros(5 + case.mech.n_reactions, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError, match="RF_CHARWISE"):
        nv.adjoint_rhs(ctx, U, T, 0.0, case.laser.as_tuple(), lam, 0.0, lam.clone(), grads)
    with pytest.raises(RuntimeError, match="RF_CHARWISE"):
        nv.create_ctx(mech, case.grid, nv.RF_FP64, nv.RF_CHARWISE | nv.RF_MAPPED)
    jet = synth.case_jet_inflow(0, 12, 8, 8)
    with pytest.raises(RuntimeError, match="RF_CHARWISE"):
        nv.create_ctx(nv.init_mechanism(jet.mech), jet.grid, nv.RF_FP64, nv.RF_CHARWISE)
