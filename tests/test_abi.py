"""The C-ABI library loads and exports every entry point its header declares, and
its host-side argument checks reject bad input before any device work.  No
compute call is made here (this runs without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2202_02319_b300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(rf_[a-z0-9_]+)\s*\(", src))
    return names


def test_library_exports_every_declared_symbol():
    from paper_2202_02319_b300 import native
    lib = ctypes.CDLL(native.LIB_PATH)
    names = _declared()
    assert len(names) >= 10
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_host_argument_checks():
    from paper_2202_02319_b300 import native as nv
    m = synth.mechanism_4sp(0)
    mech = nv.init_mechanism(m)                    # host-only packing, no device call
    assert mech.n_species == 4
    bad = synth.mechanism_4sp(0)
    bad.W = bad.W.copy()
    bad.W[1] = -1.0
    with pytest.raises(nv.ReactFlowError) as e:
        nv.init_mechanism(bad)
    assert e.value.code == nv.RF_EINVAL
    # five species: not a supported species count
    five = synth.Mechanism(["A"] * 5, np.full(5, 0.02), np.ones((5, 1)), np.zeros((5, 7)), np.zeros((5, 7)),
                           np.full(5, 1000.0), np.full(5, 2e-5), np.full(5, 0.7), np.full((5, 5), 2e-5),
                           np.zeros(0), np.zeros(0), np.zeros(0), np.zeros((0, 5), dtype=np.int64),
                           np.zeros((0, 5), dtype=np.int64), np.zeros(0, dtype=np.int32))
    with pytest.raises(nv.ReactFlowError):
        nv.init_mechanism(five)
    # grid checks happen before any allocation
    for g in (synth.Grid(0, 4, 4, 1e-4, 1e-4, 1e-4), synth.Grid(2048, 1, 1, 1e-4, 1e-4, 1e-4),
              synth.Grid(4, 4, 4, -1.0, 1e-4, 1e-4), synth.Grid(4, 4, 4, 1e-4, 1e-4, 1e-4, (0, 7, 0)),
              synth.Grid(4, 2, 4, 1e-4, 1e-4, 1e-4, (0, synth.BC_NSCBC, 0))):
        with pytest.raises(nv.ReactFlowError) as e:
            nv.create_ctx(mech, g)
        assert e.value.code == nv.RF_EINVAL
    # NSCBC: the allocation-free RHS has no context for the side settings; a null
    # context is refused before any device call
    f = ctypes.CDLL(nv.LIB_PATH).rf_rhs_noalloc
    f.restype = ctypes.c_int
    f.argtypes = [ctypes.c_void_p, ctypes.POINTER(nv.GridDesc), ctypes.c_int, ctypes.c_uint32, ctypes.c_void_p,
                  ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    gd = nv.GridDesc(8, 8, 1, 1e-4, 1e-4, 1e-4, (ctypes.c_int * 3)(synth.BC_NSCBC, 0, 0))
    assert f(mech.handle, ctypes.byref(gd), 0, 0, 16, 16, 0.0, None, 16, None) == nv.RF_EINVAL
    assert "NSCBC" in nv.last_error()
    d = nv.NscbcDesc(101325.0, 0.25, 1.0, 1.0, 1.0, 1.0, 0.0, None)
    assert nv._lib.rf_set_nscbc(None, 0, 0, ctypes.byref(d)) == nv.RF_EINVAL
    # the stored-stage adjoint entry points refuse null pointers before any device call
    assert nv._lib.rf_rk_step_stages(None, None, None, 0.0, 1e-9, None, None, None, None) == nv.RF_EINVAL
    assert "rf_rk_step_stages" in nv.last_error()
    assert nv._lib.rf_adjoint_rk_step_stored(None, None, None, 0.0, 1e-9, None, 1.0, None, None, None) == nv.RF_EINVAL
    assert "rf_adjoint_rk_step_stored" in nv.last_error()
    # more than three molecules on one side of a reaction
    m2 = synth.mechanism_4sp(0)
    m2.nu_f = m2.nu_f.copy()
    m2.nu_f[0, 0] = 4
    with pytest.raises(nv.ReactFlowError):
        nv.init_mechanism(m2)
