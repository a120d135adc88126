"""Thin Python binding of libfpclosure.so (C ABI in include/fpclosure.h).

Argument marshalling only: every step of the closure runs in the library's
CUDA kernels.  Tensors must be CUDA tensors; the call is enqueued on the
current torch stream (or the one given).  There is no CPU fallback: without
the compiled library or a GPU every entry point raises.
"""

from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import build as _build

NMOM = 30
NCOEF = 9
LU_STRIDE = 82
NDIAG = 12
NLITE = 14
NSENS = 11


def lu_doubles(n_cells: int) -> int:
    """Size (float64 entries) of the factor buffer of fp_closure_solve."""
    return (n_cells + 31) // 32 * 32 * LU_STRIDE
FP_OK, FP_ERR_ARG, FP_ERR_CUDA, FP_ERR_WORKSPACE, FP_ERR_UNSUPPORTED = 0, -1, -2, -3, -4
V_F32, V_F64 = 0, 1
PREC_FP64, PREC_FP32_MOMENTS = 0, 1
FLAG_FEW, FLAG_SINGULAR, FLAG_NONFINITE, FLAG_RANGE, FLAG_ENERGY, FLAG_FALLBACK, FLAG_ALPHA = 1, 2, 4, 8, 16, 32, 64
FALLBACK_FLAGS = FLAG_FEW | FLAG_SINGULAR | FLAG_NONFINITE
FP32_PIVOT_FLOOR = 1e-6
FP32_MIN_REGULAR = 5  # FP32-moment mode flags cells with fewer particles singular

_PREC = {"fp64": PREC_FP64, "fp32": PREC_FP32_MOMENTS, PREC_FP64: PREC_FP64, PREC_FP32_MOMENTS: PREC_FP32_MOMENTS}


class FPError(RuntimeError):
    pass


class Params(ctypes.Structure):
    _fields_ = [("eps2_hat", ctypes.c_double), ("min_particles", ctypes.c_int32),
                ("pivot_rtol", ctypes.c_double), ("surr_energy_tol", ctypes.c_double),
                ("surr_range_margin", ctypes.c_double), ("particle_offset", ctypes.c_uint64)]


class FpMlp(ctypes.Structure):
    """fp_mlp of fpclosure.h (device pointers)."""
    _fields_ = [("W", ctypes.c_void_p * 5), ("b", ctypes.c_void_p * 5),
                ("x_mu", ctypes.c_void_p), ("x_sigma", ctypes.c_void_p),
                ("y_mu", ctypes.c_void_p), ("y_sigma", ctypes.c_void_p),
                ("x_min", ctypes.c_void_p), ("x_max", ctypes.c_void_p),
                ("in_dim", ctypes.c_int32), ("hidden", ctypes.c_int32), ("depth", ctypes.c_int32),
                ("out_dim", ctypes.c_int32), ("eps2_hat", ctypes.c_double)]


_LIB = None
_LOCK = threading.Lock()
_vp, _i64, _i32, _sz, _dbl, _u64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_size_t, ctypes.c_double, ctypes.c_uint64


class StepIO(ctypes.Structure):
    """fp_step_io of fpclosure.h (host and device pointers)."""
    _fields_ = [("h_v", _vp), ("h_v_out", _vp), ("h_offsets", _vp), ("h_tau", _vp), ("h_coeffs", _vp),
                ("h_flags", _vp),
                ("d_v", _vp), ("d_v_out", _vp), ("d_offsets", _vp), ("d_tau", _vp), ("d_moments", _vp),
                ("d_m6", _vp),
                ("d_coeffs", _vp), ("d_flags", _vp), ("d_flags_v", _vp),
                ("net", ctypes.POINTER(FpMlp)), ("d_coeffs_s", _vp), ("d_flags_s", _vp), ("d_surrogate_ws", _vp),
                ("surrogate_ws_bytes", _sz),
                ("d_lu", _vp), ("d_grad_coeffs", _vp), ("d_grad_moments", _vp), ("d_grad_v", _vp)]


# name -> (restype, argtypes); the exported surface of include/fpclosure.h
SIGNATURES = {
    "fp_diagnostics": (_i32, [_vp, _vp, _vp, _i64, _dbl, _dbl, _dbl, _vp, _vp]),
    "fp_coeffs_relax": (_i32, [_vp, _vp, _i64, _dbl, _vp]),
    "fp_pipeline_create": (_i32, [ctypes.POINTER(_vp)]),
    "fp_pipeline_destroy": (None, [_vp]),
    "fp_step_host": (_i32, [_vp, ctypes.POINTER(StepIO), _i32, _i64, _i64, ctypes.POINTER(Params), _i32, _dbl,
                            _u64, _u64, _i32, _vp]),
    "fp_default_params": (None, [ctypes.POINTER(Params)]),
    "fp_status_string": (ctypes.c_char_p, [_i32]),
    "fp_last_error": (ctypes.c_char_p, []),
    "fp_version": (_i32, []),
    "fp_workspace_bytes": (_sz, [_i64, _i64, _i32, _i32]),
    "fp_closure_exact": (_i32, [_vp, _i32, _i64, _vp, _i64, _vp, ctypes.POINTER(Params), _i32,
                                _vp, _vp, _vp, _vp, _sz, _vp]),
    "fp_moments": (_i32, [_vp, _i32, _i64, _vp, _i64, _i32, _vp, _vp, _vp]),
    "fp_closure_solve": (_i32, [_vp, _vp, _i64, ctypes.POINTER(Params), _i32, _vp, _vp, _vp, _vp]),
    "fp_velocity_update": (_i32, [_vp, _vp, _i32, _i64, _vp, _i64, _vp, _vp, _vp, _vp, _dbl,
                                  ctypes.POINTER(Params), _vp, _u64, _u64, _vp, _vp, _vp]),
    "fp_closure_backward": (_i32, [_vp, _i32, _i64, _vp, _i64, _vp, ctypes.POINTER(Params), _vp, _vp, _vp, _vp,
                                   _vp, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fp_mlp_param_count": (_i64, []),
    "fp_mlp_param_offset": (_i64, [_i32, _i32]),
    "fp_surrogate_workspace_bytes": (_sz, [_i64]),
    "fp_surrogate_features": (_i32, [ctypes.POINTER(FpMlp), _vp, _i64, _vp, ctypes.POINTER(Params), _vp, _vp, _vp]),
    "fp_surrogate_training_rows": (_i32, [_vp, _vp, _vp, _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "fp_mlp_forward": (_i32, [ctypes.POINTER(FpMlp), _vp, _i64, _i32, _vp, _vp, _vp, _vp]),
    "fp_closure_surrogate": (_i32, [ctypes.POINTER(FpMlp), _vp, _i64, _vp, ctypes.POINTER(Params), _i32, _vp, _vp,
                                    _vp, _sz, _vp]),
    "fp_surrogate_loss": (_i32, [_vp, _vp, _vp, _vp, _vp, _i64, _vp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, _vp, _vp, _vp, _vp]),
    "fp_mlp_backward_workspace_bytes": (_sz, [_i64]),
    "fp_mlp_backward": (_i32, [ctypes.POINTER(FpMlp), _vp, _vp, _vp, _vp, _vp, _i64, _vp, _vp, _sz, _vp]),
    "fp_adam_step": (_i32, [_vp, _vp, _vp, _vp, _i64, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, _i64, _vp, _vp]),
    "fp_surrogate_train_step_workspace_bytes": (_sz, [_i64]),
    "fp_surrogate_train_step": (_i32, [ctypes.POINTER(FpMlp), _vp, _vp, _vp, _i64, _vp, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, _vp, _vp, _vp, _vp, _i64, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_float, ctypes.c_float, _i64, _vp, _vp, _vp, _sz,
                                       _vp]),
    "fp_closure_exact_static": (_i32, [_vp, _i32, _i64, _vp, _i64, _vp, ctypes.POINTER(Params), _i32, _vp, _vp,
                                       _vp]),
    "fp_closure_exact_static_error": (ctypes.c_char_p, []),
    "fp_moments_lite": (_i32, [_vp, _i32, _i64, _vp, _i64, _vp, _vp]),
    "fp_velocity_update_lite": (_i32, [_vp, _vp, _i32, _i64, _vp, _i64, _vp, _vp, _vp, _dbl,
                                       ctypes.POINTER(Params), _vp, _u64, _u64, _vp, _vp, _vp]),
    "fp_surrogate_sensitivity_workspace_bytes": (_sz, [_i64]),
    "fp_surrogate_sensitivity": (_i32, [ctypes.POINTER(FpMlp), _vp, _i32, _i64, _vp, ctypes.POINTER(Params), _i32,
                                        _dbl, _u64, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fp_sort_workspace_bytes": (_sz, [_i64, _i64]),
    "fp_sort_by_cell": (_i32, [_vp, _i64, _i64, _vp, _i32, _vp, _vp, _vp, _vp, _sz, _vp]),
    "fp_collision_step_workspace_bytes": (_sz, [_i64, _i64, _i32, _i32]),
    "fp_collision_step": (_i32, [_vp, _vp, _i32, _i64, _i64, _vp, ctypes.POINTER(Params), _i32,
                                 ctypes.POINTER(FpMlp), _dbl, _u64, _u64, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _sz,
                                 _vp]),
    "fp_surrogate_lite_features": (_i32, [ctypes.POINTER(FpMlp), _vp, _i64, _vp, ctypes.POINTER(Params), _vp, _vp,
                                          _vp]),
    "fp_surrogate_lite_workspace_bytes": (_sz, [_i64]),
    "fp_closure_surrogate_lite": (_i32, [ctypes.POINTER(FpMlp), _vp, _i64, _vp, ctypes.POINTER(Params), _vp, _vp,
                                         _vp, _sz, _vp]),
    "fp_selftest_wait_timeout": (_i32, [_u64, _vp, _vp, _vp]),
}

STATIC_MAX_CELLS = 32768


def fp_closure_exact_static(v, offsets, tau, params: Params | None = None, prec="fp32", coeffs_out=None,
                            flags_out=None, stream=None):
    """The exact closure with the library's built-in scratch array instead of
    caller memory (for callers that may not allocate; at most
    STATIC_MAX_CELLS cells) -> (coeffs, flags)."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    dev = offsets.device
    if coeffs_out is None:
        coeffs_out = torch.empty((n_cells, NCOEF), dtype=torch.float64, device=dev)
    if flags_out is None:
        flags_out = torch.empty((n_cells,), dtype=torch.int32, device=dev)
    _need_cuda(v, offsets, tau, coeffs_out, flags_out)
    _want_cells(n_cells, offsets, tau, None, coeffs_out, flags_out)
    p = params if params is not None else default_params()
    rc = lib().fp_closure_exact_static(_ptr(v), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(tau),
                                       ctypes.byref(p), _PREC.get(prec, prec), _ptr(coeffs_out), _ptr(flags_out),
                                       _stream(stream))
    if rc != FP_OK:
        raise FPError(f"fp_closure_exact_static: {lib().fp_status_string(rc).decode()} "
                      f"({lib().fp_closure_exact_static_error().decode()})")
    return coeffs_out, flags_out


def fp_closure_backward(v, offsets, tau, moments, coeffs, flags, grad_coeffs, grad_moments_in=None,
                        params: Params | None = None, want_grad_moments=True, want_grad_v=True,
                        grad_moments=None, grad_v=None, workspace=None, stream=None, lu=None):
    """Adjoint of the closure -> (grad_moments or None, grad_v or None).
    lu: the factors fp_closure_solve kept for the same moments (optional)."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    dev = offsets.device
    if want_grad_moments and grad_moments is None:
        grad_moments = torch.empty((n_cells, NMOM), dtype=torch.float64, device=dev)
    if want_grad_v and grad_v is None:
        grad_v = torch.empty_like(v)
    _need_cuda(v, offsets, tau, moments, coeffs, flags, grad_coeffs, grad_moments_in, grad_moments, grad_v, workspace,
               lu)
    if lu is not None and (lu.dtype != torch.float64 or lu.numel() < lu_doubles(n_cells)):
        raise FPError(f"lu must be float64 with lu_doubles(n_cells) = {lu_doubles(n_cells)} entries")
    _want_cells(n_cells, offsets, tau, moments, coeffs, flags)
    _want(grad_coeffs, "grad_coeffs", torch.float64, n_cells * NCOEF)
    _want(grad_moments_in, "grad_moments_in", torch.float64, n_cells * NMOM)
    _want(grad_moments, "grad_moments", torch.float64, n_cells * NMOM)
    _want(grad_v, "grad_v", v.dtype, 3 * n_p)
    need = workspace_bytes(n_cells, n_p, "fp64", grad_moments is not None) if grad_v is not None else 0
    if need and workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    p = params if params is not None else default_params()
    rc = lib().fp_closure_backward(_ptr(v), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(tau), ctypes.byref(p),
                                   _ptr(moments), _ptr(coeffs), _ptr(flags), _ptr(lu), _ptr(grad_coeffs),
                                   _ptr(grad_moments_in), _ptr(grad_moments), _ptr(grad_v), _ptr(workspace),
                                   ws_bytes, _stream(stream))
    _check(rc, "fp_closure_backward")
    return grad_moments, grad_v


def fp_diagnostics(moments, m6, rho=None, theta_inf=1.0, rho_inf=1.0, dg_inf=0.0, out=None, stream=None):
    """Per-cell high-order diagnostics and entropy proxies [n_cells, NDIAG]:
    R_ij / theta^2 (6), <|c|^4> / theta^2 - 15, <|c|^6> / theta^3, D_G, D_q,
    Delta s_eq, Delta s_kin,G (fpclosure.h)."""
    n_cells = moments.shape[0]
    if out is None:
        out = torch.empty((n_cells, NDIAG), dtype=torch.float64, device=moments.device)
    _need_cuda(moments, m6, rho, out)
    _want_cells(n_cells, moments=moments)
    _want(m6, "m6", torch.float64, n_cells)
    _want(rho, "rho", torch.float64, n_cells)
    _want(out, "out", torch.float64, n_cells * NDIAG)
    rc = lib().fp_diagnostics(_ptr(moments), _ptr(m6), _ptr(rho), n_cells, float(theta_inf), float(rho_inf),
                              float(dg_inf), _ptr(out), _stream(stream))
    _check(rc, "fp_diagnostics")
    return out


def fp_coeffs_relax(coeffs_new, coeffs_prev, w=0.2, stream=None):
    """coeffs_prev <- w coeffs_new + (1 - w) coeffs_prev (in place)."""
    _need_cuda(coeffs_new, coeffs_prev)
    if coeffs_new.shape != coeffs_prev.shape or coeffs_new.dtype != torch.float64:
        raise FPError("coeffs_new and coeffs_prev must be float64 of the same shape")
    _want(coeffs_prev, "coeffs_prev", torch.float64, coeffs_prev.shape[0] * NCOEF)
    rc = lib().fp_coeffs_relax(_ptr(coeffs_new), _ptr(coeffs_prev), coeffs_prev.shape[0], float(w), _stream(stream))
    _check(rc, "fp_coeffs_relax")
    return coeffs_prev


class HostStep:
    """One step of the hot path on velocities in host memory (fp_step_host):
    exact closure, optionally the learned closure and the adjoint, and the
    velocity update, with the host <-> device copies of each chunk of cells
    overlapped with the compute of the others.  Owns the full-size device
    buffers and the pipeline's streams; host tensors should be pinned.

        hs = HostStep(n_cells, n_particles, surrogate=s, adjoint=True)
        hs(h_v, h_offsets, h_tau, h_v_out, h_coeffs, h_flags, dt=0.1, seed=1, step=n)
    """

    def __init__(self, n_cells, n_particles, dtype=torch.float32, surrogate=None, adjoint=False, device=None):
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.n_cells, self.n_particles, self.dtype, self.device = n_cells, n_particles, dtype, dev
        f64 = dict(dtype=torch.float64, device=dev)
        self.d_v = torch.empty((3, n_particles), dtype=dtype, device=dev)
        self.d_v_out = torch.empty_like(self.d_v)
        self.d_offsets = torch.empty(n_cells + 1, dtype=torch.int64, device=dev)
        self.d_tau = torch.empty(n_cells, **f64)
        self.moments = torch.empty((n_cells, NMOM), **f64)
        self.m6 = torch.empty(n_cells, **f64)
        self.coeffs = torch.empty((n_cells, NCOEF), **f64)
        self.flags = torch.empty(n_cells, dtype=torch.int32, device=dev)
        self.flags_v = torch.empty_like(self.flags)
        self.surrogate = surrogate
        if surrogate is not None:
            self.coeffs_s = torch.empty_like(self.coeffs)
            self.flags_s = torch.empty_like(self.flags)
            self.surrogate_ws = torch.empty(int(lib().fp_surrogate_workspace_bytes(n_cells)), dtype=torch.uint8,
                                            device=dev)
        self.adjoint = adjoint
        if adjoint:
            self.lu = torch.empty(lu_doubles(n_cells), **f64)
            self.grad_coeffs = torch.ones((n_cells, NCOEF), **f64)
            self.grad_moments = torch.empty_like(self.moments)
            self.grad_v = torch.empty_like(self.d_v)
        h = _vp()
        _check(lib().fp_pipeline_create(ctypes.byref(h)), "fp_pipeline_create")
        self._pl = h

    def __call__(self, h_v, h_offsets, h_tau, h_v_out, h_coeffs, h_flags, dt, params: Params | None = None,
                 prec="fp32", seed=0, step=0, n_chunks=8, stream=None):
        for t in (h_v, h_offsets, h_tau, h_v_out, h_coeffs, h_flags):
            if t.is_cuda or not t.is_contiguous():
                raise FPError("fp_step_host takes contiguous host tensors")
        nc, npart = self.n_cells, self.n_particles
        _want(h_v, "h_v", self.dtype, 3 * npart)
        _want(h_v_out, "h_v_out", self.dtype, 3 * npart)
        _want(h_offsets, "h_offsets", torch.int64, nc + 1)
        _want(h_tau, "h_tau", torch.float64, nc)
        _want(h_coeffs, "h_coeffs", torch.float64, nc * NCOEF)
        _want(h_flags, "h_flags", torch.int32, nc)
        io = StepIO()
        io.h_v, io.h_v_out = h_v.data_ptr(), h_v_out.data_ptr()
        io.h_offsets, io.h_tau = h_offsets.data_ptr(), h_tau.data_ptr()
        io.h_coeffs, io.h_flags = h_coeffs.data_ptr(), h_flags.data_ptr()
        io.d_v, io.d_v_out = self.d_v.data_ptr(), self.d_v_out.data_ptr()
        io.d_offsets, io.d_tau = self.d_offsets.data_ptr(), self.d_tau.data_ptr()
        io.d_moments, io.d_coeffs = self.moments.data_ptr(), self.coeffs.data_ptr()
        io.d_m6 = self.m6.data_ptr()
        io.d_flags, io.d_flags_v = self.flags.data_ptr(), self.flags_v.data_ptr()
        net = None
        if self.surrogate is not None:
            net = self.surrogate.net()
            io.net = ctypes.pointer(net)
            io.d_coeffs_s, io.d_flags_s = self.coeffs_s.data_ptr(), self.flags_s.data_ptr()
            io.d_surrogate_ws, io.surrogate_ws_bytes = self.surrogate_ws.data_ptr(), self.surrogate_ws.numel()
        if self.adjoint:
            io.d_lu = self.lu.data_ptr()
            io.d_grad_coeffs, io.d_grad_moments = self.grad_coeffs.data_ptr(), self.grad_moments.data_ptr()
            io.d_grad_v = self.grad_v.data_ptr()
        p = params if params is not None else default_params()
        rc = lib().fp_step_host(self._pl, ctypes.byref(io), _vdtype(self.d_v), self.n_particles, self.n_cells,
                                ctypes.byref(p), _PREC.get(prec, prec), float(dt), int(seed), int(step),
                                int(n_chunks), _stream(stream))
        _check(rc, "fp_step_host")
        return h_v_out, h_coeffs, h_flags

    def close(self):
        if getattr(self, "_pl", None):
            lib().fp_pipeline_destroy(self._pl)
            self._pl = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libfpclosure.so (building it in-tree first if it is stale)."""
    global _LIB
    with _LOCK:
        if _LIB is None:
            path = _build.build()
            if not os.path.exists(path):
                raise FPError(f"libfpclosure.so missing at {path}")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.restype = res
                fn.argtypes = args
            _LIB = L
    return _LIB


def default_params(**kw) -> Params:
    p = Params()
    lib().fp_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def _check(rc: int, what: str):
    if rc != FP_OK:
        L = lib()
        raise FPError(f"{what}: {L.fp_status_string(rc).decode()} ({L.fp_last_error().decode()})")


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and (not isinstance(t, torch.Tensor) or not t.is_cuda):
            raise FPError("arguments must be CUDA tensors (there is no CPU path)")
        if t is not None and not t.is_contiguous():
            raise FPError("arguments must be contiguous")


def _vdtype(v):
    if v.dtype == torch.float32:
        return V_F32
    if v.dtype == torch.float64:
        return V_F64
    raise FPError(f"velocity dtype {v.dtype} (float32 or float64 expected)")


def _nv(v):
    """Particle count of velocities [3, n_particles] (or the flat SoA array
    of 3 n_particles entries)."""
    _vdtype(v)
    if (v.dim() == 2 and v.shape[0] != 3) or v.numel() % 3:
        raise FPError(f"velocities must be [3, n_particles], not {tuple(v.shape)}")
    return v.numel() // 3


def _want(t, name, dtype, numel):
    """Checks a tensor before its pointer crosses the C ABI, which takes plain
    pointers: the dtype the call reads or writes, and at least the entries it
    touches.  None passes (the entry point treats it as absent)."""
    if t is None:
        return
    if t.dtype != dtype:
        raise FPError(f"{name} must be {dtype}, not {t.dtype}")
    if t.numel() < numel:
        raise FPError(f"{name} must hold at least {numel} entries, not {t.numel()}")


def _want_cells(n_cells, offsets=None, tau=None, moments=None, coeffs=None, flags=None, stride=NMOM):
    """The per-cell arrays of a call on n_cells cells."""
    _want(offsets, "offsets", torch.int64, n_cells + 1)
    _want(tau, "tau", torch.float64, n_cells)
    _want(moments, "moments", torch.float64, n_cells * stride)
    _want(coeffs, "coeffs", torch.float64, n_cells * NCOEF)
    _want(flags, "flags", torch.int32, n_cells)


def workspace_bytes(n_cells, n_particles, prec="fp32", moments_out_given=False) -> int:
    return int(lib().fp_workspace_bytes(n_cells, n_particles, _PREC.get(prec, prec), int(bool(moments_out_given))))


def fp_closure_exact(v, offsets, tau, params: Params | None = None, prec="fp32", moments_out=None,
                     coeffs_out=None, flags_out=None, workspace=None, want_moments=True, stream=None):
    """The exact closure.  v [3, n_p] (f32/f64), offsets [n_cells+1] int64,
    tau [n_cells] f64 -> (moments [n_cells, 30] or None, coeffs [n_cells, 9],
    flags [n_cells])."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    dev = offsets.device
    if want_moments and moments_out is None:
        moments_out = torch.empty((n_cells, NMOM), dtype=torch.float64, device=dev)
    if coeffs_out is None:
        coeffs_out = torch.empty((n_cells, NCOEF), dtype=torch.float64, device=dev)
    if flags_out is None:
        flags_out = torch.empty((n_cells,), dtype=torch.int32, device=dev)
    _need_cuda(v, offsets, tau, moments_out, coeffs_out, flags_out, workspace)
    _want_cells(n_cells, offsets, tau, moments_out, coeffs_out, flags_out)
    need = workspace_bytes(n_cells, n_p, prec, moments_out is not None)
    if need and workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    ws_bytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    p = params if params is not None else default_params()
    rc = lib().fp_closure_exact(_ptr(v), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(tau), ctypes.byref(p),
                                _PREC.get(prec, prec), _ptr(moments_out), _ptr(coeffs_out), _ptr(flags_out),
                                _ptr(workspace), ws_bytes, _stream(stream))
    _check(rc, "fp_closure_exact")
    return moments_out, coeffs_out, flags_out


def fp_moments(v, offsets, prec="fp32", moments_out=None, stream=None, m6_out=None):
    """Per-cell moment vectors [n_cells, 30] (f64); m6_out (float64
    [n_cells], optional) receives <|c|^6> for a one-pass velocity update."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    if moments_out is None:
        moments_out = torch.empty((n_cells, NMOM), dtype=torch.float64, device=offsets.device)
    _need_cuda(v, offsets, moments_out, m6_out)
    _want_cells(n_cells, offsets, moments=moments_out)
    _want(m6_out, "m6_out", torch.float64, n_cells)
    rc = lib().fp_moments(_ptr(v), _vdtype(v), n_p, _ptr(offsets), n_cells, _PREC.get(prec, prec),
                          _ptr(moments_out), _ptr(m6_out), _stream(stream))
    _check(rc, "fp_moments")
    return moments_out


def fp_moments_lite(v, offsets, out=None, stream=None):
    """LITE moment vectors [n_cells, NLITE] (f64): N, U (3), theta, u_ij
    (6), b_i = <c_i |c|^2> (3), from FP32 compensated sums."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    if out is None:
        out = torch.empty((n_cells, NLITE), dtype=torch.float64, device=offsets.device)
    _need_cuda(v, offsets, out)
    _want_cells(n_cells, offsets)
    _want(out, "out", torch.float64, n_cells * NLITE)
    rc = lib().fp_moments_lite(_ptr(v), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(out), _stream(stream))
    _check(rc, "fp_moments_lite")
    return out


def fp_surrogate_training_rows(moments, tau, coeffs=None, lite=None, lite_inputs=False, raw=True, targets=True,
                               aux=True, stream=None):
    """(raw [n, 32], targets [n, 16], aux [n, 16]) FP32 rows for training the
    learned closure, from the library's kernels (None for outputs not asked
    for): the unstandardised inputs as the inference kernels form them (full
    set from `moments`, or LITE set from `lite` and tau), the dimensionless
    targets of `coeffs`, the loss's auxiliary moments of `moments`."""
    n = tau.numel()
    dev = tau.device
    r = torch.empty((n, 32), dtype=torch.float32, device=dev) if raw else None
    t = torch.empty((n, 16), dtype=torch.float32, device=dev) if targets else None
    x = torch.empty((n, 16), dtype=torch.float32, device=dev) if aux else None
    _need_cuda(moments, tau, coeffs, lite, r, t, x)
    _want_cells(n, None, tau, moments, coeffs)
    if lite is not None:
        _want_cells(n, None, None, lite, None, None, stride=NLITE)
    rc = lib().fp_surrogate_training_rows(_ptr(moments), _ptr(lite), _ptr(coeffs), _ptr(tau), n,
                                          1 if lite_inputs else 0, _ptr(r), _ptr(t), _ptr(x), _stream(stream))
    _check(rc, "fp_surrogate_training_rows")
    return r, t, x


def fp_sort_by_cell(cell_of, n_cells, v=None, v_sorted=None, perm_out=None, offsets_out=None, workspace=None,
                    stream=None):
    """Stable order of the particles by cell -> (perm int32 [n_p], offsets
    int64 [n_cells + 1], v_sorted or None).  Cell indices outside
    [0, n_cells) go behind the last cell."""
    n_p = cell_of.numel()
    dev = cell_of.device
    if cell_of.dtype != torch.int32:
        raise FPError("cell_of must be int32")
    perm = perm_out if perm_out is not None else torch.empty(n_p, dtype=torch.int32, device=dev)
    off = offsets_out if offsets_out is not None else torch.empty(n_cells + 1, dtype=torch.int64, device=dev)
    if v is not None and v_sorted is None:
        v_sorted = torch.empty_like(v)
    need = int(lib().fp_sort_workspace_bytes(n_p, n_cells))
    ws = workspace if workspace is not None else torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    _need_cuda(cell_of, perm, off, v, v_sorted, ws)
    _want(perm, "perm_out", torch.int32, n_p)
    _want(off, "offsets_out", torch.int64, n_cells + 1)
    if v is not None:
        if _nv(v) != n_p:
            raise FPError("v must hold the velocities of the cell_of particles")
        _want(v_sorted, "v_sorted", v.dtype, 3 * n_p)
    rc = lib().fp_sort_by_cell(_ptr(cell_of), n_p, n_cells, _ptr(v), _vdtype(v) if v is not None else 0,
                               _ptr(v_sorted), _ptr(perm), _ptr(off), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "fp_sort_by_cell")
    return perm, off, v_sorted


def fp_collision_step(cell_of, v, n_cells, tau, dt, params: Params | None = None, prec="fp32", net_lite=None,
                      seed=0, step=0, v_out=None, perm_out=None, offsets_out=None, coeffs_out=None, flags_out=None,
                      moments_out=None, workspace=None, stream=None):
    """Sort by cell, closure (exact, or the learned one on LITE inputs when
    net_lite -- an FpMlp -- is given) and velocity update in one call ->
    (v_out in sorted order, perm, offsets, coeffs, flags)."""
    n_p = cell_of.numel()
    dev = v.device
    lite = net_lite is not None
    v_out = v_out if v_out is not None else torch.empty_like(v)
    perm = perm_out if perm_out is not None else torch.empty(n_p, dtype=torch.int32, device=dev)
    off = offsets_out if offsets_out is not None else torch.empty(n_cells + 1, dtype=torch.int64, device=dev)
    y = coeffs_out if coeffs_out is not None else torch.empty((n_cells, 9), dtype=torch.float64, device=dev)
    fl = flags_out if flags_out is not None else torch.empty(n_cells, dtype=torch.int32, device=dev)
    need = int(lib().fp_collision_step_workspace_bytes(n_p, n_cells, _vdtype(v), int(lite)))
    ws = workspace if workspace is not None else torch.empty(need, dtype=torch.uint8, device=dev)
    _need_cuda(cell_of, v, tau, v_out, perm, off, y, fl, moments_out, ws)
    _want(cell_of, "cell_of", torch.int32, n_p)
    if _nv(v) != n_p:
        raise FPError("v must hold the velocities of the cell_of particles")
    _want(v_out, "v_out", v.dtype, 3 * n_p)
    _want(perm, "perm_out", torch.int32, n_p)
    _want_cells(n_cells, off, tau, moments_out, y, fl, stride=NLITE if lite else NMOM)
    p = params if params is not None else default_params()
    rc = lib().fp_collision_step(_ptr(cell_of), _ptr(v), _vdtype(v), n_p, n_cells, _ptr(tau), ctypes.byref(p),
                                 _PREC.get(prec, prec), ctypes.byref(net_lite) if lite else None, float(dt),
                                 int(seed), int(step), _ptr(v_out), _ptr(perm), _ptr(off), _ptr(y), _ptr(fl),
                                 _ptr(moments_out), _ptr(ws), ws.numel(), _stream(stream))
    _check(rc, "fp_collision_step")
    return v_out, perm, off, y, fl


def fp_closure_solve(moments, tau, params: Params | None = None, prec="fp32", coeffs_out=None, flags_out=None,
                     stream=None, lu_out=None):
    """Assembly + pivoted FP64 solve from moment vectors -> (coeffs, flags).
    lu_out: float64 of lu_doubles(n_cells) entries receiving the factors
    the adjoint can reuse (fp_closure_backward(lu=...)), tiled by 32 cells."""
    n_cells = moments.shape[0]
    dev = moments.device
    if coeffs_out is None:
        coeffs_out = torch.empty((n_cells, NCOEF), dtype=torch.float64, device=dev)
    if flags_out is None:
        flags_out = torch.empty((n_cells,), dtype=torch.int32, device=dev)
    _need_cuda(moments, tau, coeffs_out, flags_out, lu_out)
    _want_cells(n_cells, None, tau, moments, coeffs_out, flags_out)
    if lu_out is not None and (lu_out.dtype != torch.float64 or lu_out.numel() < lu_doubles(n_cells)):
        raise FPError(f"lu_out must be float64 with lu_doubles(n_cells) = {lu_doubles(n_cells)} entries")
    p = params if params is not None else default_params()
    rc = lib().fp_closure_solve(_ptr(moments), _ptr(tau), n_cells, ctypes.byref(p), _PREC.get(prec, prec),
                                _ptr(coeffs_out), _ptr(flags_out), _ptr(lu_out), _stream(stream))
    _check(rc, "fp_closure_solve")
    return coeffs_out, flags_out


def fp_velocity_update(v, offsets, moments, coeffs, tau, flags, dt, params: Params | None = None, xi=None,
                       seed=0, step=0, alpha_out=None, stream=None, v_out=None, m6=None):
    """One velocity update (Eqs. update_vel / update_N / update_alpha), in
    place or into v_out (same shape and dtype, not overlapping v).  flags is
    read and updated; returns (updated velocities, alpha_out, flags).  With
    m6 (fp_moments' m6_out of the same velocities) the particles are read
    once."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    _need_cuda(v, offsets, moments, coeffs, tau, flags, xi, alpha_out, v_out, m6)
    if v_out is not None and (v_out.dtype != v.dtype or v_out.numel() != v.numel()):
        raise FPError("v_out must be an array of v's shape and dtype")
    _want(xi, "xi", v.dtype, 3 * n_p)
    _want_cells(n_cells, offsets, tau, moments, coeffs, flags)
    _want(alpha_out, "alpha_out", torch.float64, n_cells)
    _want(m6, "m6", torch.float64, n_cells)
    p = params if params is not None else default_params()
    rc = lib().fp_velocity_update(_ptr(v), _ptr(v_out), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(moments),
                                  _ptr(m6),
                                  _ptr(coeffs), _ptr(tau), float(dt), ctypes.byref(p), _ptr(xi), int(seed), int(step),
                                  _ptr(alpha_out), _ptr(flags), _stream(stream))
    _check(rc, "fp_velocity_update")
    return (v if v_out is None else v_out), alpha_out, flags


def fp_velocity_update_lite(v, offsets, lite, coeffs, tau, flags, dt, params: Params | None = None, xi=None,
                            seed=0, step=0, alpha_out=None, stream=None, v_out=None):
    """fp_velocity_update from LITE moment vectors [n_cells, NLITE] (alpha's
    cell averages summed over the particles)."""
    n_cells = offsets.numel() - 1
    n_p = _nv(v)
    _need_cuda(v, offsets, lite, coeffs, tau, flags, xi, alpha_out, v_out)
    if v_out is not None and (v_out.dtype != v.dtype or v_out.numel() != v.numel()):
        raise FPError("v_out must be an array of v's shape and dtype")
    _want(xi, "xi", v.dtype, 3 * n_p)
    _want_cells(n_cells, offsets, tau, lite, coeffs, flags, stride=NLITE)
    _want(alpha_out, "alpha_out", torch.float64, n_cells)
    p = params if params is not None else default_params()
    rc = lib().fp_velocity_update_lite(_ptr(v), _ptr(v_out), _vdtype(v), n_p, _ptr(offsets), n_cells, _ptr(lite),
                                       _ptr(coeffs), _ptr(tau), float(dt), ctypes.byref(p), _ptr(xi), int(seed),
                                       int(step), _ptr(alpha_out), _ptr(flags), _stream(stream))
    _check(rc, "fp_velocity_update_lite")
    return (v if v_out is None else v_out), alpha_out, flags


def fp_selftest_wait_timeout(limit_ns=1_000_000, stream=None):
    """Self-test of the library's bounded mbarrier wait: a wait on a barrier
    nothing completes, limited to limit_ns -> (status, waited_ns); status 0
    means the wait gave up as it should."""
    dev = torch.device("cuda", torch.cuda.current_device())
    status = torch.full((1,), -1, dtype=torch.int32, device=dev)
    waited = torch.zeros(1, dtype=torch.int64, device=dev)
    _check(lib().fp_selftest_wait_timeout(int(limit_ns), _ptr(status), _ptr(waited), _stream(stream)),
           "fp_selftest_wait_timeout")
    return int(status.item()), int(waited.item())

