"""The allocation-free RHS entry point (rf_rhs_noalloc), called through the C
ABI, gives the same dU/dt as the context-based rf_rhs on two calls in a row.

This entry point exists for callers that cannot allocate device memory: a host
framework whose caching allocator already holds the device's memory budget,
and latency-critical loops where cudaMalloc / cudaFree may synchronise the
device.  Its scratch is a fixed 16 MiB device array shared by all calls.  The
file sorts last so that a run stopping at the first failure has run every
other test before this one."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2202_02319_b300 import synth

pytestmark = pytest.mark.gpu


def _lib():
    from paper_2202_02319_b300 import native as nv
    lib = ctypes.CDLL(nv.LIB_PATH)
    f = lib.rf_rhs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(nv.GridDesc), ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.POINTER(nv.Laser), ctypes.c_void_p, ctypes.c_void_p]
    return nv, f


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_noalloc_rhs_matches_context_rhs_on_two_calls(precision):
    nv, f = _lib()
    case = synth.case_jet(0, 16)
    case.laser.t0 = 2e-8
    ns = case.mech.n_species
    n = case.grid.ncells
    mech = nv.init_mechanism(case.mech)
    ctx = nv.create_ctx(mech, case.grid, precision)
    prim = torch.as_tensor(case.prim, dtype=torch.float64).reshape(5 + ns, n).cuda()
    U = torch.empty((ns + 4, n), dtype=torch.float64, device="cuda")
    T0 = torch.empty(n, dtype=torch.float64, device="cuda")
    nv.init_state(ctx, prim, U, T0)
    ref = torch.empty_like(U)
    Tr = T0.clone()
    nv.rhs(ctx, U, Tr, 0.0, case.laser.as_tuple(), ref)
    nv.check(ctx)
    g = case.grid
    gd = nv.GridDesc(g.nx, g.ny, g.nz, g.dx, g.dy, g.dz, (ctypes.c_int * 3)(*g.bc))
    las = nv.Laser(*case.laser.as_tuple())
    stream = torch.cuda.current_stream().cuda_stream
    scale = ref.abs().amax(1)
    for call in range(2):
        out = torch.full_like(U, float("nan"))
        T = T0.clone()
        rc = f(mech.handle, ctypes.byref(gd), precision, 0, U.data_ptr(), T.data_ptr(), 0.0, ctypes.byref(las),
               out.data_ptr(), stream)
        assert rc == 0, nv.last_error()
        err = ((out - ref).abs().amax(1) / torch.where(scale > 0, scale, torch.ones_like(scale))).max().item()
        assert err <= 1e-12, (call, err)
        assert torch.equal(T, Tr)


def test_noalloc_rejects_grids_beyond_its_scratch():
    nv, f = _lib()
    m = synth.mechanism_9sp(0)
    mech = nv.init_mechanism(m)
    gd = nv.GridDesc(64, 64, 64, 1e-4, 1e-4, 1e-4, (ctypes.c_int * 3)(0, 0, 0))
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = f(mech.handle, ctypes.byref(gd), 0, 0, dummy.data_ptr(), dummy.data_ptr(), 0.0, None, dummy.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
    assert rc == nv.RF_EINVAL and "maximum" in nv.last_error()


def test_noalloc_rejects_charwise():
    """RF_CHARWISE runs through a context only."""
    nv, f = _lib()
    mech = nv.init_mechanism(synth.mechanism_9sp(0))
    gd = nv.GridDesc(8, 8, 8, 1e-4, 1e-4, 1e-4, (ctypes.c_int * 3)(0, 0, 0))
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc = f(mech.handle, ctypes.byref(gd), 0, nv.RF_CHARWISE, dummy.data_ptr(), dummy.data_ptr(), 0.0, None,
           dummy.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert rc == nv.RF_EINVAL and "RF_CHARWISE" in nv.last_error()
