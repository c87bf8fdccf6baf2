"""ctypes binding and numpy drivers for the plain C oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: used by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``.  Never imported by the library.

Everything here is FP64 except ``forward_f32``, the same sweep evaluated
in FP32 (``oracle_f32.c``).  Arrays are halo-padded C-order numpy arrays of
shape (nz+2R, ny+2R, nx+2R); coefficient stacks have shape (k, nz+2R,
ny+2R, nx+2R).  The update definitions, kind numbers and the time-state
convention are documented in ``oracle.c`` (paper Sect. 3.1, Fig. 1).
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA = 1, 2, 3, 4, 5, 6
RADIUS = {J7_CONST: 1, J7_VAR: 1, W25_CONST: 4, W25_VAR: 4, J25_VAR: 4, W25_ALPHA: 4}
NUM_ARRAYS = {J7_CONST: 0, J7_VAR: 7, W25_CONST: 0, W25_VAR: 13, J25_VAR: 13, W25_ALPHA: 1}
NUM_WEIGHTS = {J7_CONST: 2, J7_VAR: 0, W25_CONST: 6, W25_VAR: 0, J25_VAR: 0, W25_ALPHA: 5}
SECOND_ORDER = {J7_CONST: False, J7_VAR: False, W25_CONST: True, W25_VAR: True,
                J25_VAR: False, W25_ALPHA: True}

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "oracle.c")
_SRC32 = os.path.join(_HERE, "oracle_f32.c")
_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return os.path.join(_BUILD, "liboracle.so")


def build(force: bool = False) -> str:
    """Compile ``oracle.c`` and ``oracle_f32.c`` into ``_build/liboracle.so`` with gcc.

    -ffp-contract=off keeps every multiply and add separately rounded so the
    oracle gives identical bits on x86_64 and aarch64 hosts.
    """
    out = lib_path()
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_SRC32))
    if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
        return out
    os.makedirs(_BUILD, exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, _SRC32]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _open(path):
    lib = ctypes.CDLL(path)
    i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
    lib.oracle_forward.argtypes = [i32, i64, i64, i64, i32, dp, dp, dp, dp, i64, dp, i64, i32]
    lib.oracle_forward.restype = i32
    lib.oracle_adjoint.argtypes = [i32, i64, i64, i64, i32, dp, dp, dp, dp, i64, dp, dp, i64,
                                   dp, i32]
    lib.oracle_adjoint.restype = i32
    if hasattr(lib, "oracle_forward_f32"):   # absent from the planted-mistake copies of oracle.c
        lib.oracle_forward_f32.argtypes = [i32, i64, i64, i64, i32, dp, dp, dp, i32, dp, i64, dp, i64, i32]
        lib.oracle_forward_f32.restype = i32
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _open(build())
    return _lib


@contextlib.contextmanager
def swapped_library(path):
    """Run the drivers against another build of the oracle source (used by the
    tests that plant a mistake in a copy of ``oracle.c``)."""
    global _lib
    _load()
    saved = _lib
    _lib = _open(path)
    try:
        yield
    finally:
        _lib = saved


def compile_variant(source_text: str, out_path: str) -> str:
    """Compile a (modified) copy of the oracle source with the same flags."""
    src = out_path + ".c"
    with open(src, "w") as f:
        f.write(source_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    "-fPIC", "-shared", "-o", out_path, src], check=True)
    return out_path


def compile_variant_f32(f32_text: str, out_path: str) -> str:
    """Compile ``oracle.c`` with a (modified) copy of ``oracle_f32.c``."""
    src = out_path + "_f32.c"
    with open(src, "w") as f:
        f.write(f32_text)
    subprocess.run(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
                    "-fPIC", "-shared", "-o", out_path, _SRC, src], check=True)
    return out_path


def source_text() -> str:
    with open(_SRC) as f:
        return f.read()


def source_text_f32() -> str:
    with open(_SRC32) as f:
        return f.read()


def _ptr(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"], "oracle arrays must be C-contiguous float64"
    return a.ctypes.data_as(ctypes.c_void_p)


def _dims(u, R):
    pz, py, px = u.shape
    return px - 2 * R, py - 2 * R, pz - 2 * R


def _weights(kind, w):
    if NUM_WEIGHTS[kind] == 0:
        return None
    w = np.ascontiguousarray(np.asarray(w, dtype=np.float64))
    assert w.shape == (NUM_WEIGHTS[kind],), f"kind {kind} takes {NUM_WEIGHTS[kind]} weights"
    return w


def _arrays(kind, W, shape):
    if NUM_ARRAYS[kind] == 0:
        return None
    W = np.ascontiguousarray(W, dtype=np.float64)
    assert W.shape == (NUM_ARRAYS[kind],) + tuple(shape)
    return W


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def forward(kind, u_prev, u, w=None, W=None, T=1, rcv_z=None, threads=1):
    """Advance (u_prev, u) by T steps of the naive sweep.

    Returns (u_prev, u, trace): new arrays holding (u^{T-1}, u^T), and, when
    ``rcv_z`` (zero-based interior z index) is given, the receiver trace
    [T, ny, nx] with trace[t] = u^{t+1} on that plane.
    """
    R = RADIUS[kind]
    a = np.array(u_prev, dtype=np.float64, order="C", copy=True)
    b = np.array(u, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = _dims(b, R)
    wv, Wv = _weights(kind, w), _arrays(kind, W, b.shape)
    trace = np.zeros((T, ny, nx)) if rcv_z is not None else None
    st = _load().oracle_forward(kind, nx, ny, nz, R, _ptr(a), _ptr(b), _ptr(wv), _ptr(Wv), int(T),
                                _ptr(trace), int(rcv_z or 0), int(threads))
    if st != 0:
        raise ValueError(f"oracle_forward failed with status {st}")
    return a, b, trace


def forward_f32(kind, u_prev, u, w=None, W=None, T=1, rcv_z=None, threads=1):
    """The FP32 evaluation of ``forward`` (oracle_f32.c): the inputs are
    rounded to float32 once, every update is evaluated in float32 in the
    FP64 oracle's order of terms.  Returns float64 arrays holding the float32
    results (u^{T-1}, u^T, trace)."""
    R = RADIUS[kind]
    a = np.array(u_prev, dtype=np.float32, order="C", copy=True)
    b = np.array(u, dtype=np.float32, order="C", copy=True)
    nx, ny, nz = _dims(b, R)
    wv = _weights(kind, w)
    Wv = None
    if NUM_ARRAYS[kind]:
        Wv = np.ascontiguousarray(W, dtype=np.float32)
        assert Wv.shape == (NUM_ARRAYS[kind],) + b.shape
    trace = np.zeros((T, ny, nx), dtype=np.float32) if rcv_z is not None else None
    p32 = (lambda x: None if x is None else x.ctypes.data_as(ctypes.c_void_p))
    st = _load().oracle_forward_f32(kind, nx, ny, nz, R, p32(a), p32(b), _ptr(wv),
                                    0 if wv is None else len(wv), p32(Wv), int(T), p32(trace),
                                    int(rcv_z or 0), int(threads))
    if st != 0:
        raise ValueError(f"oracle_forward_f32 failed with status {st}")
    return (a.astype(np.float64), b.astype(np.float64),
            trace.astype(np.float64) if trace is not None else None)


def adjoint(kind, lam_next, lam, w=None, W=None, T=1, states=None, residual=None, rcv_z=None,
            grad=None, threads=1):
    """Run T adjoint steps; see the adjoint section of ``oracle.c``.

    ``states`` is [T, pz, py, px] with states[i] = u^{m-T+i}; ``residual`` is
    [T, ny, nx] with residual[i] the receiver residual at level m-T+i;
    ``grad`` (k, pz, py, px) is accumulated in place.  Returns new arrays
    (lam_next, lam) = (lam^{m-T+1}, lam^{m-T}).
    """
    R = RADIUS[kind]
    a = np.array(lam_next, dtype=np.float64, order="C", copy=True)
    b = np.array(lam, dtype=np.float64, order="C", copy=True)
    nx, ny, nz = _dims(b, R)
    wv, Wv = _weights(kind, w), _arrays(kind, W, b.shape)
    if states is not None:
        states = np.ascontiguousarray(states, dtype=np.float64)
        assert states.shape == (T,) + b.shape
    if residual is not None:
        residual = np.ascontiguousarray(residual, dtype=np.float64)
        assert residual.shape == (T, ny, nx)
    if grad is not None:
        assert grad.dtype == np.float64 and grad.flags["C_CONTIGUOUS"]
        assert grad.shape == (NUM_ARRAYS[kind],) + b.shape
    st = _load().oracle_adjoint(kind, nx, ny, nz, R, _ptr(a), _ptr(b), _ptr(wv), _ptr(Wv), int(T),
                                _ptr(states), _ptr(residual), int(rcv_z or 0), _ptr(grad), int(threads))
    if st != 0:
        raise ValueError(f"oracle_adjoint failed with status {st}")
    return a, b


def receiver_loss(trace, d):
    """0.5 * sum over steps and receiver plane of (trace - d)^2, in FP64."""
    r = np.asarray(trace, dtype=np.float64) - np.asarray(d, dtype=np.float64)
    return 0.5 * float(np.sum(r * r)), r


def loss_and_gradient(kind, u0, W, d, T, rcv_z, w=None, threads=1):
    """Receiver-misfit loss and its gradient w.r.t. u0 and the coefficient arrays.

    Forward: u^{-1} = u^0 = u0 (zero initial velocity for wave kinds), T steps,
    loss = 0.5 * sum_{t=1..T} |P u^t - d^t|^2 with P the receiver plane.
    All states are kept (no checkpointing: this is the plain reference).
    Returns (loss, dL/du0, dL/dW).
    """
    R = RADIUS[kind]
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    states = np.empty((T + 1,) + u0.shape)
    states[0] = u0
    p, c = u0.copy(), u0.copy()
    trace = np.empty((T,) + (u0.shape[1] - 2 * R, u0.shape[2] - 2 * R))
    for t in range(T):
        p, c, tr = forward(kind, p, c, w, W, 1, rcv_z=rcv_z, threads=threads)
        states[t + 1] = c
        trace[t] = tr[0]
    loss, r = receiver_loss(trace, d)
    # lam^T = g^T, lam^{T+1} = 0; residual for levels 0..T-1 (level 0 has no misfit term)
    lam = np.zeros_like(u0)
    lam_next = np.zeros_like(u0)
    nz = u0.shape[0] - 2 * R
    zp = rcv_z + R
    lam[zp, R:-R, R:-R] = r[T - 1]
    res = np.zeros((T,) + r.shape[1:])
    res[1:] = r[:T - 1]
    grad = np.zeros((NUM_ARRAYS[kind],) + u0.shape) if NUM_ARRAYS[kind] else None
    assert 0 <= rcv_z < nz
    lam_next, lam = adjoint(kind, lam_next, lam, w, W, T, states=states[:T], residual=res,
                            rcv_z=rcv_z, grad=grad, threads=threads)
    if SECOND_ORDER[kind]:
        # u^{-1} is tied to u^0: dL/du0 = lam^0 - lam^1
        du0 = lam - lam_next
    else:
        du0 = lam
    return loss, du0, grad
