"""Thin Python binding of the C ABI in include/reactflow.h.

Argument marshalling only: every step of the method runs in the CUDA library.
Functions keep the C names without the `rf_` prefix.  Device arrays are torch
CUDA tensors (float64, contiguous) passed as raw pointers on the current torch
stream.  If the shared library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "lib", "libreactflow.so")

RF_OK, RF_EINVAL, RF_ENEWTON, RF_ENONFINITE, RF_ERANGE, RF_ECUDA, RF_ETIMEOUT, RF_ENOMEM = 0, -1, -2, -3, -4, -5, -6, -7
RF_FP64, RF_MIXED = 0, 1
RF_NO_INVISCID, RF_NO_VISCOUS, RF_NO_CHEMISTRY, RF_NO_LASER, RF_TENO6, RF_MAPPED, RF_CHARWISE = 1, 2, 4, 8, 16, 32, 64
RF_BC_PERIODIC, RF_BC_EXTRAPOLATE, RF_BC_NSCBC = 0, 1, 2
CODE_NAMES = {0: "RF_OK", -1: "RF_EINVAL", -2: "RF_ENEWTON", -3: "RF_ENONFINITE", -4: "RF_ERANGE",
              -5: "RF_ECUDA", -6: "RF_ETIMEOUT", -7: "RF_ENOMEM"}

if not os.path.exists(LIB_PATH):
    raise ImportError(f"CUDA library not built: {LIB_PATH} is missing (run paper_2202_02319_b300/build.py)")
_lib = ctypes.CDLL(LIB_PATH)

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)


class MechDesc(ctypes.Structure):
    _fields_ = [("n_species", ctypes.c_int), ("n_reactions", ctypes.c_int), ("W", _dp), ("nasa_low", _dp),
                ("nasa_high", _dp), ("T_mid", _dp), ("mu_ref", _dp), ("mu_exp", _dp), ("D_ref", _dp),
                ("A", _dp), ("b", _dp), ("Theta", _dp), ("nu_f", _ip), ("nu_r", _ip), ("reversible", _ip),
                ("rxn_type", _ip), ("efficiency", _dp), ("A0", _dp), ("b0", _dp), ("Theta0", _dp), ("troe", _dp)]


class GridDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double),
                ("dy", ctypes.c_double), ("dz", ctypes.c_double), ("bc", ctypes.c_int * 3)]


class Laser(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("E", "x0", "y0", "z0", "sigma_r", "t0", "sigma_t")]


class NscbcDesc(ctypes.Structure):
    _fields_ = [(k, ctypes.c_double) for k in ("p_inf", "sigma", "eta_u", "eta_T", "eta_t", "eta_Y", "length")] + \
        [("target", ctypes.c_void_p)]


class Diag(ctypes.Structure):
    _fields_ = [("total", ctypes.c_double * 32), ("heat_release", ctypes.c_double), ("max_T", ctypes.c_double),
                ("nv", ctypes.c_int)]


_vp = ctypes.c_void_p
_sigs = {
    "rf_last_error": (ctypes.c_char_p, []),
    "rf_init_mechanism": (ctypes.c_int, [ctypes.POINTER(MechDesc), ctypes.POINTER(_vp)]),
    "rf_free_mechanism": (None, [_vp]),
    "rf_create_ctx": (ctypes.c_int, [_vp, ctypes.POINTER(GridDesc), ctypes.c_int, ctypes.c_uint32, ctypes.POINTER(_vp)]),
    "rf_free_ctx": (None, [_vp]),
    "rf_ctx_workspace_bytes": (ctypes.c_size_t, [_vp]),
    "rf_init_state": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "rf_rhs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(Laser), _vp, _vp]),
    "rf_rk_step": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Laser), _vp, _vp]),
    "rf_rk_step_host": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(Laser), _vp, _vp]),
    "rf_set_option": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_double]),
    "rf_set_nscbc": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.POINTER(NscbcDesc)]),
    "rf_set_nodes": (ctypes.c_int, [_vp, _vp, _vp]),
    "rf_profile_read": (ctypes.c_int, [_vp, _dp, _ip, ctypes.c_int]),
    "rf_probe_peak": (ctypes.c_int, [ctypes.c_int, _dp, _vp]),
    "rf_probe_math": (ctypes.c_int, [ctypes.c_int, _vp, _vp, _vp, ctypes.c_longlong, _vp]),
    "rf_adjoint_rhs": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.POINTER(Laser), _vp, ctypes.c_double, _vp,
                                      _vp, _vp]),
    "rf_rk_step_objective": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Laser), _dp,
                                            _vp]),
    "rf_adjoint_rk_step": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Laser),
                                          ctypes.c_double, _vp, _vp, _vp]),
    "rf_rk_step_stages": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double, ctypes.POINTER(Laser), _dp,
                                         _vp, _vp]),
    "rf_adjoint_rk_step_stored": (ctypes.c_int, [_vp, _vp, _vp, ctypes.c_double, ctypes.c_double,
                                                 ctypes.POINTER(Laser), ctypes.c_double, _vp, _vp, _vp]),
    "rf_ensemble_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                          ctypes.POINTER(Laser), _vp, ctypes.POINTER(_vp)]),
    "rf_ensemble_free": (None, [_vp]),
    "rf_ensemble_set_option": (ctypes.c_int, [_vp, ctypes.c_char_p, ctypes.c_double]),
    "rf_run_ensemble": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.POINTER(ctypes.c_int32), _vp]),
    "rf_ensemble_autotune": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_int), _vp]),
    "rf_status": (ctypes.c_int, [_vp, _vp, ctypes.POINTER(ctypes.c_longlong)]),
    "rf_diagnostics": (ctypes.c_int, [_vp, _vp, _vp, ctypes.POINTER(Diag), _vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


class ReactFlowError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = _lib.rf_last_error().decode(errors="replace")
        super().__init__(f"{where}: {CODE_NAMES.get(code, code)}: {msg}")


def _check(code: int, where: str):
    if code != RF_OK:
        raise ReactFlowError(code, where)


def _ptr(t) -> int:
    if t is None:
        return None
    import torch
    if not (t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CUDA tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def last_error() -> str:
    return _lib.rf_last_error().decode(errors="replace")


class Mechanism:
    """Device copy of a mechanism (rf_init_mechanism / rf_free_mechanism)."""

    def __init__(self, m):
        ns, nr = m.n_species, m.n_reactions
        keep = []

        def d(a):
            a = np.ascontiguousarray(a, dtype=np.float64)
            keep.append(a)
            return a.ctypes.data_as(_dp)

        def i(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(a)
            return a.ctypes.data_as(_ip)
        desc = MechDesc(ns, nr, d(m.W), d(m.nasa_low), d(m.nasa_high), d(m.T_mid), d(m.mu_ref), d(m.mu_exp),
                        d(m.D_ref), d(m.A if nr else np.zeros(1)), d(m.b if nr else np.zeros(1)),
                        d(m.Theta if nr else np.zeros(1)), i(m.nu_f if nr else np.zeros(1)),
                        i(m.nu_r if nr else np.zeros(1)), i(m.reversible if nr else np.zeros(1)))
        rt = getattr(m, "rxn_type", None)
        if rt is not None and nr and np.any(np.asarray(rt) != 0):
            desc.rxn_type = i(rt)
            desc.efficiency = d(m.efficiency)
            desc.A0, desc.b0, desc.Theta0 = d(m.A0), d(m.b0), d(m.Theta0)
            desc.troe = d(m.troe)
        h = _vp()
        _check(_lib.rf_init_mechanism(ctypes.byref(desc), ctypes.byref(h)), "rf_init_mechanism")
        self.handle = h
        self.n_species = ns
        self.n_reactions = nr

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.rf_free_mechanism(self.handle)
            self.handle = None


def init_mechanism(m) -> Mechanism:
    return Mechanism(m)


class Context:
    """Solver context for one grid (rf_create_ctx / rf_free_ctx)."""

    def __init__(self, mech: Mechanism, grid, precision: int = RF_FP64, flags: int = 0):
        g = GridDesc(grid.nx, grid.ny, grid.nz, grid.dx, grid.dy, grid.dz, (ctypes.c_int * 3)(*grid.bc))
        h = _vp()
        _check(_lib.rf_create_ctx(mech.handle, ctypes.byref(g), precision, flags, ctypes.byref(h)), "rf_create_ctx")
        self.handle = h
        self.mech = mech
        self.grid = grid
        self.precision = precision
        self.flags = flags
        self.n = grid.nx * grid.ny * grid.nz
        self.nv = mech.n_species + 4
        self.nscbc_targets = {}          # (axis, side) -> inflow target tensor the library reads

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.rf_free_ctx(self.handle)
            self.handle = None

    @property
    def workspace_bytes(self) -> int:
        return int(_lib.rf_ctx_workspace_bytes(self.handle))


def create_ctx(mech: Mechanism, grid, precision: int = RF_FP64, flags: int = 0) -> Context:
    return Context(mech, grid, precision, flags)


def _laser(las) -> Optional[Laser]:
    if las is None:
        return None
    t = las.as_tuple() if hasattr(las, "as_tuple") else tuple(las)
    return Laser(*[float(v) for v in t])


def init_state(ctx: Context, prim, U, T, stream=None):
    _check(_lib.rf_init_state(ctx.handle, _ptr(prim), _ptr(U), _ptr(T), _stream(stream)), "rf_init_state")


def rhs(ctx: Context, U, T, t: float, laser, dUdt, stream=None):
    L = _laser(laser)
    _check(_lib.rf_rhs(ctx.handle, _ptr(U), _ptr(T), float(t), ctypes.byref(L) if L else None, _ptr(dUdt),
                       _stream(stream)), "rf_rhs")


def rk_step(ctx: Context, U, T, t_dev, dt_fixed: float = 0.0, cfl: float = 0.5, laser=None, dt_dev=None, stream=None):
    L = _laser(laser)
    _check(_lib.rf_rk_step(ctx.handle, _ptr(U), _ptr(T), _ptr(t_dev), float(dt_fixed), float(cfl),
                           ctypes.byref(L) if L else None, _ptr(dt_dev), _stream(stream)), "rf_rk_step")


def _hptr(t) -> int:
    if t is None:
        return None
    import torch
    if not (t.device.type == "cpu" and t.dtype == torch.float64 and t.is_contiguous()):
        raise ValueError("expected a contiguous float64 CPU tensor")
    return t.data_ptr()


def rk_step_host(ctx: Context, U_in, T_in, U_out, T_out, t_dev, dt_fixed: float = 0.0, cfl: float = 0.5, laser=None,
                 dt_dev=None, stream=None):
    """One SSP-RK3 step on host tensors (pinned for overlap): U_in, T_in copied in by chunks
    overlapping the first stage, the new state written to U_out (and T_out if given).
    Asynchronous on the stream, like the device-buffer step."""
    L = _laser(laser)
    _check(_lib.rf_rk_step_host(ctx.handle, _hptr(U_in), _hptr(T_in), _hptr(U_out), _hptr(T_out), _ptr(t_dev),
                                float(dt_fixed), float(cfl), ctypes.byref(L) if L else None, _ptr(dt_dev),
                                _stream(stream)), "rf_rk_step_host")


def set_option(ctx: Context, key: str, value: float):
    _check(_lib.rf_set_option(ctx.handle, key.encode(), float(value)), "rf_set_option")


def set_nodes(ctx: Context, nodes, stream=None):
    """Node coordinates of an RF_MAPPED context (rf_set_nodes): a contiguous float64
    CUDA tensor [3, nz + 1, ny + 1, nx + 1]; synchronous."""
    g = ctx.grid
    if tuple(nodes.shape) != (3, g.nz + 1, g.ny + 1, g.nx + 1):
        raise ValueError(f"nodes must have shape (3, {g.nz + 1}, {g.ny + 1}, {g.nx + 1})")
    _check(_lib.rf_set_nodes(ctx.handle, _ptr(nodes), _stream(stream)), "rf_set_nodes")


def set_nscbc(ctx: Context, axis: int, side: int, p_inf: float = 101325.0, sigma: float = 0.25, eta_u: float = 1.0,
              eta_T: float = 1.0, eta_t: float = 1.0, eta_Y: float = 1.0, length: float = 0.0, target=None):
    """One end of an NSCBC axis (rf_set_nscbc): an outflow when target is None, else an
    inflow relaxing towards target, a contiguous float64 CUDA tensor [4 + Ns, plane]
    (u, v, w, T, Y_s) that the context keeps a reference to while the side is set."""
    if target is not None:
        import torch
        if not (target.is_cuda and target.dtype == torch.float64 and target.is_contiguous()):
            raise ValueError("target must be a contiguous float64 CUDA tensor")
    d = NscbcDesc(float(p_inf), float(sigma), float(eta_u), float(eta_T), float(eta_t), float(eta_Y), float(length),
                  _ptr(target) if target is not None else None)
    _check(_lib.rf_set_nscbc(ctx.handle, int(axis), int(side), ctypes.byref(d)), "rf_set_nscbc")
    if target is not None:
        ctx.nscbc_targets[(axis, side)] = target
    else:
        ctx.nscbc_targets.pop((axis, side), None)


def probe_peak(kind: int, stream=None) -> float:
    """Measured FMA throughput in TFLOP/s (kind 0: FP64, 1: FP32)."""
    v = ctypes.c_double(0.0)
    _check(_lib.rf_probe_peak(int(kind), ctypes.byref(v), _stream(stream)), "rf_probe_peak")
    return v.value


def probe_exp_pair(x, ep, em, stream=None):
    """ep = exp(x), em = exp(-x) by the kernels' FP64 exponential pair (device tensors)."""
    _check(_lib.rf_probe_math(0, _ptr(x), _ptr(ep), _ptr(em), int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_log(x, y, stream=None):
    """y = ln x by the kernels' FP64 logarithm (device tensors)."""
    _check(_lib.rf_probe_math(1, _ptr(x), _ptr(y), None, int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_exp(x, y, stream=None):
    """y = exp(x) by the kernels' single FP64 exponential (device tensors)."""
    _check(_lib.rf_probe_math(2, _ptr(x), _ptr(y), None, int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_exp_pair_mixed(x, ep, em, stream=None):
    """ep = exp(x), em = exp(-x) by the mixed path's FP64 exponential pair (device tensors)."""
    _check(_lib.rf_probe_math(5, _ptr(x), _ptr(ep), _ptr(em), int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_log_mixed(x, y, stream=None):
    """y = ln x by the mixed path's FP64 logarithm (device tensors)."""
    _check(_lib.rf_probe_math(6, _ptr(x), _ptr(y), None, int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_d2f(x, y, y2, stream=None):
    """y = the kernels' binary32 rounding of x, y2 = the hardware's (float64 device tensors)."""
    _check(_lib.rf_probe_math(3, _ptr(x), _ptr(y), _ptr(y2), int(x.numel()), _stream(stream)), "rf_probe_math")


def probe_f2d(x, y, y2, stream=None):
    """Low 32 bits of each x hold a binary32 pattern f: y = the kernels' widening of f,
    y2 = the hardware's (float64 device tensors)."""
    _check(_lib.rf_probe_math(4, _ptr(x), _ptr(y), _ptr(y2), int(x.numel()), _stream(stream)), "rf_probe_math")


PROF_CLASSES = ("cell_state", "sweep_x", "sweep_y", "sweep_z", "other")


def profile_read(ctx: Context) -> dict:
    """{class: (total_ms, launches)} since profiling was enabled or last read."""
    ms = (ctypes.c_double * 5)()
    ln = (ctypes.c_int * 5)()
    _check(_lib.rf_profile_read(ctx.handle, ms, ln, 5), "rf_profile_read")
    return {k: (ms[i], ln[i]) for i, k in enumerate(PROF_CLASSES)}


def status(ctx: Context, stream=None):
    """(code, cell) of the device-side status; clears it."""
    cell = ctypes.c_longlong(-1)
    code = _lib.rf_status(ctx.handle, _stream(stream), ctypes.byref(cell))
    return code, cell.value


def check(ctx: Context, stream=None):
    code, _ = status(ctx, stream)
    _check(code, "rf_status")


def diagnostics(ctx: Context, U, T, stream=None) -> dict:
    d = Diag()
    _check(_lib.rf_diagnostics(ctx.handle, _ptr(U), _ptr(T), ctypes.byref(d), _stream(stream)), "rf_diagnostics")
    return {"total": np.array(d.total[:d.nv]), "heat_release": d.heat_release, "max_T": d.max_T}


ENS_LOOP, ENS_BATCHED, ENS_GRAPH, ENS_PERSISTENT = 0, 1, 2, 3


class Ensemble:
    """Members (contexts with their states, lasers and times) advanced together
    (rf_ensemble_create / rf_ensemble_free)."""

    def __init__(self, ctxs, Us, Ts, lasers, t_dev):
        n = len(ctxs)
        self._keep = (list(ctxs), list(Us), list(Ts), t_dev)
        hs = (_vp * n)(*[c.handle.value for c in ctxs])
        us = (_vp * n)(*[_ptr(u) for u in Us])
        ts = (_vp * n)(*[_ptr(t) for t in Ts])
        ls = (Laser * n)(*[(_laser(l) if l is not None else Laser()) for l in lasers]) if lasers is not None else None
        h = _vp()
        _check(_lib.rf_ensemble_create(hs, n, us, ts, ls, _ptr(t_dev), ctypes.byref(h)), "rf_ensemble_create")
        self.handle = h
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None):
            _lib.rf_ensemble_free(self.handle)
            self.handle = None


def ensemble_create(ctxs, Us, Ts, lasers, t_dev) -> Ensemble:
    return Ensemble(ctxs, Us, Ts, lasers, t_dev)


def ensemble_set_option(e: Ensemble, key: str, value: float):
    _check(_lib.rf_ensemble_set_option(e.handle, key.encode(), float(value)), "rf_ensemble_set_option")


def run_ensemble(e: Ensemble, nsteps: int, mode: int = ENS_GRAPH, cfl: float = 0.5, dt_fixed: float = 0.0,
                 stream=None, raise_on_error: bool = True):
    """Returns (code, per-member codes)."""
    st = (ctypes.c_int32 * e.n)()
    code = _lib.rf_run_ensemble(e.handle, int(nsteps), int(mode), float(cfl), float(dt_fixed), st, _stream(stream))
    if raise_on_error:
        _check(code, "rf_run_ensemble")
    return code, list(st)


def ensemble_autotune(e: Ensemble, mode: int = ENS_GRAPH, cfl: float = 0.5, stream=None) -> int:
    seg = ctypes.c_int(0)
    _check(_lib.rf_ensemble_autotune(e.handle, int(mode), float(cfl), ctypes.byref(seg), _stream(stream)),
           "rf_ensemble_autotune")
    return seg.value


def adjoint_rhs(ctx: Context, U, T, t: float, laser, lam_dUdt, w_hrr: float, lam_U, grad_params, stream=None):
    """lam_U += (dR/dU)^T lam_dUdt + w_hrr dH/dU; grad_params += the parameter part."""
    L = _laser(laser)
    _check(_lib.rf_adjoint_rhs(ctx.handle, _ptr(U), _ptr(T), float(t), ctypes.byref(L) if L else None,
                               _ptr(lam_dUdt) if lam_dUdt is not None else None, float(w_hrr), _ptr(lam_U),
                               _ptr(grad_params), _stream(stream)), "rf_adjoint_rhs")


def rk_step_objective(ctx: Context, U, T, t: float, dt: float, laser=None, stream=None, want_J: bool = True) -> float:
    """Advances U, T by one RK3 step; returns this step's dt sum_k b_k H(U^(k))
    (0.0 without evaluating H when want_J is False)."""
    L = _laser(laser)
    J = ctypes.c_double(0.0)
    _check(_lib.rf_rk_step_objective(ctx.handle, _ptr(U), _ptr(T), float(t), float(dt), ctypes.byref(L) if L else None,
                                     ctypes.byref(J) if want_J else None, _stream(stream)), "rf_rk_step_objective")
    return J.value


def adjoint_rk_step(ctx: Context, Un, Tn, t: float, dt: float, laser, w_hrr: float, lam, grad_params, stream=None):
    L = _laser(laser)
    _check(_lib.rf_adjoint_rk_step(ctx.handle, _ptr(Un), _ptr(Tn), float(t), float(dt), ctypes.byref(L) if L else None,
                                   float(w_hrr), _ptr(lam), _ptr(grad_params), _stream(stream)), "rf_adjoint_rk_step")


def stages_size(ctx: Context) -> int:
    """Doubles of the stages buffer rk_step_stages fills: (2 (Ns + 4) + 3) N."""
    return (2 * ctx.nv + 3) * ctx.n


def rk_step_stages(ctx: Context, U, T, t: float, dt: float, laser, stages, stream=None, want_J: bool = False) -> float:
    """rk_step_objective that also keeps the step's stage inputs in `stages` (a CUDA
    float64 tensor of stages_size(ctx) values) for adjoint_rk_step_stored."""
    if stages.numel() < stages_size(ctx) or stages.element_size() != 8 or not stages.is_cuda:
        raise ValueError("stages: a CUDA float64 tensor of stages_size(ctx) values")
    L = _laser(laser)
    J = ctypes.c_double(0.0)
    _check(_lib.rf_rk_step_stages(ctx.handle, _ptr(U), _ptr(T), float(t), float(dt), ctypes.byref(L) if L else None,
                                  ctypes.byref(J) if want_J else None, _ptr(stages), _stream(stream)), "rf_rk_step_stages")
    return J.value


def adjoint_rk_step_stored(ctx: Context, Un, stages, t: float, dt: float, laser, w_hrr: float, lam, grad_params,
                           stream=None):
    """adjoint_rk_step from the stage inputs rk_step_stages kept (their temperatures are
    overwritten)."""
    if stages.numel() < stages_size(ctx):
        raise ValueError("stages: fewer than stages_size(ctx) values")
    L = _laser(laser)
    _check(_lib.rf_adjoint_rk_step_stored(ctx.handle, _ptr(Un), _ptr(stages), float(t), float(dt),
                                          ctypes.byref(L) if L else None, float(w_hrr), _ptr(lam), _ptr(grad_params),
                                          _stream(stream)), "rf_adjoint_rk_step_stored")
