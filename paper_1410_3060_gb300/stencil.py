"""Thin ctypes binding of libstencil.so (include/stencil.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Tensors are torch CUDA tensors (PyTorch supplies device memory and
streams); their data pointers and the current CUDA stream are passed to the
C functions of the same names.  There is no CPU fallback: if the library is
not built, the first call raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import build as _build

J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA = 1, 2, 3, 4, 5, 6
F64, F32 = 0, 1
OPT_TIME_BLOCK, OPT_SCHEME, OPT_SCRATCH_BYTES, OPT_GRAD_BATCH, OPT_VARIANT, OPT_GRAPH = 1, 2, 3, 4, 5, 6
OPT_WAIT_LIMIT, OPT_TEST_SKIP_COPY = 7, 8
OPT_ADJ_TIME_BLOCK = 9
OK, EINVAL, EUNSUPPORTED, ENOMEM, ECUDA, ETIMEOUT = 0, -1, -2, -3, -4, -5
RADIUS = {J7_CONST: 1, J7_VAR: 1, W25_CONST: 4, W25_VAR: 4, J25_VAR: 4, W25_ALPHA: 4}
NUM_ARRAYS = {J7_CONST: 0, J7_VAR: 7, W25_CONST: 0, W25_VAR: 13, J25_VAR: 13, W25_ALPHA: 1}
NUM_WEIGHTS = {J7_CONST: 2, J7_VAR: 0, W25_CONST: 6, W25_VAR: 0, J25_VAR: 0, W25_ALPHA: 5}
SECOND_ORDER = {J7_CONST: False, J7_VAR: False, W25_CONST: True, W25_VAR: True, J25_VAR: False,
                W25_ALPHA: True}

# every symbol include/stencil.h declares
EXPORTED = ("stencil_plan", "stencil_plan_set", "stencil_plan_get", "stencil_plan_destroy",
            "stencil_forward", "stencil_forward_states", "stencil_adjoint", "stencil_axpby",
            "stencil_misfit", "stencil_misfit_static", "stencil_fill_zero", "stencil_schedule", "stencil_fma_peak",
            "stencil_strerror", "stencil_last_cuda_error", "stencil_wait_timeouts", "stencil_check",
            "stencil_pass_info", "stencil_debug_bad_store", "stencil_adjoint_schedule")
MISFIT_STATIC_MAX_ELEMS = 8192 * 2048

_lock = threading.Lock()
_lib = None


class StencilError(RuntimeError):
    def __init__(self, fn, status):
        msg = lib().stencil_strerror(status).decode()
        extra = ""
        if status == -4:
            extra = f" (cudaError {lib().stencil_last_cuda_error()})"
        super().__init__(f"{fn} failed: {msg} [{status}]{extra}")
        self.status = status


class _Coeffs(ctypes.Structure):
    _fields_ = [("w", ctypes.POINTER(ctypes.c_double)), ("nw", ctypes.c_int32), ("arrays", ctypes.c_void_p)]


def library_path() -> str:
    """The library this process loads: the in-tree build, or the file named
    by the environment variable STENCIL_LIBRARY (e.g. the debug build)."""
    return os.environ.get("STENCIL_LIBRARY") or _build.LIB


def lib():
    """Load libstencil.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            path = library_path()
            if not os.path.exists(path):
                raise RuntimeError(f"libstencil.so is not built ({path}); run __graft_entry__.build()")
            L = ctypes.CDLL(path)
            i64, i32, vp, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
            L.stencil_plan.argtypes = [ctypes.POINTER(vp), i32, i64, i64, i64, i32, i32]
            L.stencil_plan_set.argtypes = [vp, i32, i64]
            L.stencil_plan_get.argtypes = [vp, i32, ctypes.POINTER(i64)]
            L.stencil_plan_destroy.argtypes = [vp]
            L.stencil_plan_destroy.restype = None
            L.stencil_forward.argtypes = [vp, vp, vp, ctypes.POINTER(_Coeffs), i64, vp, vp, i64]
            L.stencil_adjoint.argtypes = [vp, vp, vp, ctypes.POINTER(_Coeffs), i64, vp, ctypes.POINTER(vp), vp,
                                          i64, vp]
            L.stencil_misfit.argtypes = [vp, vp, vp, i64, vp, vp, vp]
            L.stencil_forward_states.argtypes = [vp, vp, vp, ctypes.POINTER(_Coeffs), i64, ctypes.POINTER(vp), vp,
                                                 vp, i64]
            L.stencil_misfit_static.argtypes = [i32, vp, vp, i64, vp, vp, vp]
            L.stencil_fill_zero.argtypes = [vp, i64, vp]
            L.stencil_axpby.argtypes = [vp, i64, ctypes.c_double, vp, ctypes.c_double, vp, vp, vp]
            L.stencil_schedule.argtypes = [i32, i32, i64, i32, ctypes.POINTER(ctypes.c_int32), i64,
                                           ctypes.POINTER(i64)]
            L.stencil_fma_peak.argtypes = [i32, vp, dp, dp]
            L.stencil_strerror.argtypes = [i32]
            L.stencil_strerror.restype = ctypes.c_char_p
            L.stencil_last_cuda_error.argtypes = []
            L.stencil_wait_timeouts.argtypes = [ctypes.POINTER(i64)]
            L.stencil_check.argtypes = [vp, vp]
            L.stencil_pass_info.argtypes = [i32, i32, i32, i32, i32, ctypes.POINTER(i64)]
            L.stencil_adjoint_schedule.argtypes = [i64, i32, i32, ctypes.POINTER(i64), i64, ctypes.POINTER(i64)]
            L.stencil_debug_bad_store.argtypes = [vp, ctypes.POINTER(i64)]
            for fn in ("stencil_plan", "stencil_plan_set", "stencil_plan_get", "stencil_forward",
                       "stencil_forward_states", "stencil_adjoint", "stencil_axpby", "stencil_misfit",
                       "stencil_misfit_static", "stencil_fill_zero",
                       "stencil_schedule", "stencil_fma_peak", "stencil_last_cuda_error", "stencil_wait_timeouts",
                       "stencil_check", "stencil_pass_info", "stencil_debug_bad_store"):
                getattr(L, fn).restype = i32
            _lib = L
    return _lib


def _check(fn, status):
    if status != 0:
        raise StencilError(fn, status)


def _stream_handle(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def schedule(kind: int, T: int, b: int, dtype: int = F32):
    """The pass/copy program stencil_forward runs (host-only query)."""
    n = ctypes.c_int64(0)
    _check("stencil_schedule", lib().stencil_schedule(kind, dtype, T, b, None, 0, ctypes.byref(n)))
    buf = (ctypes.c_int32 * (6 * max(1, n.value)))()
    _check("stencil_schedule", lib().stencil_schedule(kind, dtype, T, b, buf, n.value, ctypes.byref(n)))
    return [tuple(buf[6 * i:6 * i + 6]) for i in range(n.value)]


def adjoint_schedule(T: int, grad_batch: int, levels: int = 1):
    """The host program stencil_adjoint runs with a gradient in batches of
    grad_batch steps and `levels` levels per pass (host-only query): a list
    of (op, a, b) -- (0, b, 0) wait for gradient batch b - 2, (1, j, n) the
    sweep of steps j .. j+n-1, (2, b, k) gradient batch b of k steps."""
    n = ctypes.c_int64(0)
    _check("stencil_adjoint_schedule", lib().stencil_adjoint_schedule(T, grad_batch, levels, None, 0,
                                                                      ctypes.byref(n)))
    buf = (ctypes.c_int64 * (3 * max(1, n.value)))()
    _check("stencil_adjoint_schedule", lib().stencil_adjoint_schedule(T, grad_batch, levels, buf, n.value,
                                                                      ctypes.byref(n)))
    return [tuple(buf[3 * i:3 * i + 3]) for i in range(n.value)]


def misfit_static(trace, d, residual, loss, stream=None):
    """stencil_misfit_static: the receiver misfit without a plan or any device
    allocation (partial sums in the library's static device array)."""
    import torch
    if trace.dtype not in (torch.float64, torch.float32):
        raise ValueError(f"trace: float64 or float32 expected, got {trace.dtype}")
    dtype = F64 if trace.dtype == torch.float64 else F32
    for name, t in (("d", d), ("residual", residual)):
        if t.dtype != trace.dtype or t.shape != trace.shape or not t.is_contiguous() or not t.is_cuda:
            raise ValueError(f"{name}: expected a contiguous CUDA tensor like trace")
    if not trace.is_contiguous() or not trace.is_cuda:
        raise ValueError("trace: contiguous CUDA tensor expected")
    if loss.dtype != torch.float64 or not loss.is_cuda or loss.numel() < 1:
        raise ValueError("loss: CUDA float64 tensor with at least one element")
    _check("stencil_misfit_static", lib().stencil_misfit_static(dtype, _ptr(trace), _ptr(d), int(trace.numel()),
                                                                _ptr(residual), _ptr(loss), _stream_handle(stream)))


def fill_zero(t, stream=None):
    """stencil_fill_zero: zero a contiguous CUDA tensor (asynchronous memset)."""
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("fill_zero: contiguous CUDA tensor expected")
    _check("stencil_fill_zero", lib().stencil_fill_zero(_ptr(t), int(t.numel() * t.element_size()),
                                                        _stream_handle(stream)))


def pass_info(kind: int, dtype: int, levels: int, scheme: int, variant: int):
    """stencil_pass_info: on-chip resources of a pass kernel configuration, or
    None where the library does not describe that family."""
    buf = (ctypes.c_int64 * 6)()
    st = lib().stencil_pass_info(kind, dtype, levels, scheme, variant, buf)
    if st == EUNSUPPORTED:
        return None
    _check("stencil_pass_info", st)
    return {"smem_bytes": buf[0], "threads": buf[1], "computed": (buf[2], buf[3]), "owned": (buf[4], buf[5])}


def fma_peak(dtype: int, stream=None):
    """(flops/s, SM clock Hz) of FP64 (dtype 0) or FP32 (1) FMA chains."""
    f, c = ctypes.c_double(0), ctypes.c_double(0)
    _check("stencil_fma_peak", lib().stencil_fma_peak(dtype, _stream_handle(stream), ctypes.byref(f),
                                                      ctypes.byref(c)))
    return f.value, c.value


def wait_timeouts() -> int:
    """stencil_wait_timeouts: bounded device waits that gave up (0 when healthy)."""
    n = ctypes.c_int64(0)
    _check("stencil_wait_timeouts", lib().stencil_wait_timeouts(ctypes.byref(n)))
    return n.value


class Plan:
    """A stencil plan (stencil_plan): kind, interior size, dtype."""

    def __init__(self, kind: int, nx: int, ny: int, nz: int, dtype: int = F64, radius: int | None = None):
        self.kind, self.n, self.dtype = kind, (nx, ny, nz), dtype
        self.R = RADIUS[kind] if radius is None else radius
        h = ctypes.c_void_p()
        _check("stencil_plan", lib().stencil_plan(ctypes.byref(h), kind, nx, ny, nz, self.R, dtype))
        self._h = h

    @property
    def padded_shape(self):
        nx, ny, nz = self.n
        R = self.R
        return (nz + 2 * R, ny + 2 * R, nx + 2 * R)

    def torch_dtype(self):
        import torch
        return torch.float64 if self.dtype == F64 else torch.float32

    def set(self, option: int, value: int):
        _check("stencil_plan_set", lib().stencil_plan_set(self._h, option, value))

    def get(self, option: int) -> int:
        v = ctypes.c_int64(0)
        _check("stencil_plan_get", lib().stencil_plan_get(self._h, option, ctypes.byref(v)))
        return v.value

    def check(self, stream=None):
        """stencil_check: wait for the plan's work on ``stream`` and raise
        StencilError (status ETIMEOUT) if a bounded device wait gave up since
        the previous check."""
        _check("stencil_check", lib().stencil_check(self._h, _stream_handle(stream)))

    def debug_bad_store(self):
        """stencil_debug_bad_store: first out-of-interior store index of the
        plan's sweeps (-1: none); None in the normal build."""
        v = ctypes.c_int64(0)
        status = lib().stencil_debug_bad_store(self._h, ctypes.byref(v))
        if status == EUNSUPPORTED:
            return None
        _check("stencil_debug_bad_store", status)
        return v.value

    def close(self):
        if getattr(self, "_h", None):
            lib().stencil_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _coeffs(self, w, W):
        c = _Coeffs()
        keep = []
        if w is not None:
            arr = (ctypes.c_double * len(w))(*[float(v) for v in w])
            keep.append(arr)
            c.w = ctypes.cast(arr, ctypes.POINTER(ctypes.c_double))
            c.nw = len(w)
        if W is not None:
            self._check_tensor(W, (NUM_ARRAYS[self.kind],) + self.padded_shape, "W")
            c.arrays = W.data_ptr()
        return c, keep

    def _check_tensor(self, t, shape, name):
        if not t.is_cuda or t.dtype != self.torch_dtype() or not t.is_contiguous() or tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name}: expected contiguous CUDA {self.torch_dtype()} of shape {shape}, "
                             f"got {t.dtype} {tuple(t.shape)} on {t.device}")

    def forward(self, u_prev, u, w=None, W=None, T=1, trace=None, rcv_z=0, stream=None):
        """stencil_forward: advance (u_prev, u) in place by T steps."""
        self._check_tensor(u_prev, self.padded_shape, "u_prev")
        self._check_tensor(u, self.padded_shape, "u")
        if trace is not None:
            self._check_tensor(trace, (T, self.n[1], self.n[0]), "trace")
        c, keep = self._coeffs(w, W)
        _check("stencil_forward", lib().stencil_forward(self._h, _ptr(u_prev), _ptr(u), ctypes.byref(c), int(T),
                                                        _stream_handle(stream), _ptr(trace), int(rcv_z)))
        del keep

    def forward_states(self, u_prev, u, w=None, W=None, states=(), trace=None, rcv_z=0, stream=None):
        """stencil_forward_states: states[t] <- u^{t+1} for t < len(states); inputs read only."""
        T = len(states)
        self._check_tensor(u_prev, self.padded_shape, "u_prev")
        self._check_tensor(u, self.padded_shape, "u")
        for s_ in states:
            self._check_tensor(s_, self.padded_shape, "state")
        if trace is not None:
            self._check_tensor(trace, (T, self.n[1], self.n[0]), "trace")
        arr = (ctypes.c_void_p * max(1, T))(*[s_.data_ptr() for s_ in states])
        c, keep = self._coeffs(w, W)
        _check("stencil_forward_states", lib().stencil_forward_states(
            self._h, _ptr(u_prev), _ptr(u), ctypes.byref(c), int(T), ctypes.cast(arr, ctypes.POINTER(ctypes.c_void_p)),
            _stream_handle(stream), _ptr(trace), int(rcv_z)))
        del keep

    def axpby(self, alpha, x, beta, y, out, stream=None):
        """stencil_axpby: out = alpha x + beta y (same-shape tensors of the plan dtype)."""
        for name, t in (("x", x), ("y", y), ("out", out)):
            self._check_tensor(t, tuple(x.shape), name)
        _check("stencil_axpby", lib().stencil_axpby(self._h, int(x.numel()), float(alpha), _ptr(x), float(beta), _ptr(y),
                                                    _ptr(out), _stream_handle(stream)))

    def adjoint(self, lam_next, lam, w=None, W=None, T=1, fwd_states=None, residual=None, rcv_z=0, grad=None,
                stream=None):
        """stencil_adjoint: T adjoint steps on (lam_next, lam) in place.
        ``fwd_states``: list of T tensors u^{m-T+i}; ``grad``: FP64 tensor
        (k, pz, py, px) accumulated in place."""
        import torch
        self._check_tensor(lam_next, self.padded_shape, "lam_next")
        self._check_tensor(lam, self.padded_shape, "lam")
        if residual is not None:
            self._check_tensor(residual, (T, self.n[1], self.n[0]), "residual")
        states = None
        if fwd_states is not None:
            if len(fwd_states) != T:
                raise ValueError("fwd_states must hold T tensors")
            for s in fwd_states:
                self._check_tensor(s, self.padded_shape, "fwd_state")
            states = (ctypes.c_void_p * max(1, T))(*[s.data_ptr() for s in fwd_states])
        if grad is not None:
            if (not grad.is_cuda or grad.dtype != torch.float64 or not grad.is_contiguous()
                    or tuple(grad.shape) != (NUM_ARRAYS[self.kind],) + self.padded_shape):
                raise ValueError("grad: expected contiguous CUDA float64 (k, pz, py, px)")
        c, keep = self._coeffs(w, W)
        _check("stencil_adjoint", lib().stencil_adjoint(
            self._h, _ptr(lam_next), _ptr(lam), ctypes.byref(c), int(T), _stream_handle(stream),
            ctypes.cast(states, ctypes.POINTER(ctypes.c_void_p)) if states is not None else None,
            _ptr(residual), int(rcv_z), _ptr(grad)))
        del keep

    def misfit(self, trace, d, residual, loss, stream=None):
        """stencil_misfit: residual = trace - d, loss[0] = 0.5 sum residual^2 (FP64)."""
        import torch
        T = trace.shape[0]
        for name, t in (("trace", trace), ("d", d), ("residual", residual)):
            self._check_tensor(t, (T, self.n[1], self.n[0]), name)
        if not loss.is_cuda or loss.dtype != torch.float64 or loss.numel() < 1:
            raise ValueError("loss: CUDA float64 tensor with at least one element")
        _check("stencil_misfit", lib().stencil_misfit(self._h, _ptr(trace), _ptr(d), int(T), _ptr(residual),
                                                      _ptr(loss), _stream_handle(stream)))
