"""Host-side checks of the C ABI (no GPU needed): the library loads, exports
every function include/stencil.h declares, rejects bad arguments without a
device, and its time-loop program leaves (u^{T-1}, u^T) in (u_prev, u)."""
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def st():
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def declared_functions():
    src = open(os.path.join(ROOT, "include", "stencil.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(stencil_[a-z_0-9]+)\s*\(", src)))


def test_header_and_binding_agree(st):
    assert declared_functions() == sorted(st.EXPORTED)


def test_library_exports_every_declared_symbol(st):
    L = st.lib()
    for name in declared_functions():
        assert hasattr(L, name), name


def test_strerror_and_invalid_arguments(st):
    L = st.lib()
    assert L.stencil_strerror(0) == b"ok"
    assert L.stencil_strerror(-1) == b"invalid argument"
    import ctypes
    h = ctypes.c_void_p()
    # bad radius for the kind, bad dtype, bad size: rejected on the host
    assert L.stencil_plan(ctypes.byref(h), 1, 8, 8, 8, 4, 0) == -1
    assert L.stencil_plan(ctypes.byref(h), 1, 8, 8, 8, 1, 7) == -1
    assert L.stencil_plan(ctypes.byref(h), 1, 0, 8, 8, 1, 0) == -1
    assert L.stencil_plan(ctypes.byref(h), 9, 8, 8, 8, 1, 0) == -1
    n = ctypes.c_int64()
    assert L.stencil_schedule(1, 1, -1, 1, None, 0, ctypes.byref(n)) == -1
    assert L.stencil_schedule(1, 1, 4, 0, None, 0, ctypes.byref(n)) == -1
    assert L.stencil_schedule(1, 5, 4, 1, None, 0, ctypes.byref(n)) == -1
    assert L.stencil_strerror(-5) == b"a bounded device wait gave up"
    assert L.stencil_check(None, None) == -1


class _FakeTensor:
    """Stands in for a CUDA tensor in the host-side argument checks."""

    def __init__(self, dtype, shape=(4, 3), cuda=True, n=None):
        self.dtype, self.shape, self.is_cuda = dtype, shape, cuda
        self._n = n if n is not None else int(np.prod(shape))

    def is_contiguous(self):
        return True

    def numel(self):
        return self._n


def test_misfit_static_rejects_other_dtypes_and_empty_loss(st):
    """Only float64 / float32 traces (the kernel reads 4 or 8 bytes per
    element) and a loss tensor with room for the result are accepted; the
    checks run before any library call."""
    import torch
    for dt in (torch.float16, torch.bfloat16, torch.int32):
        t = _FakeTensor(dt)
        with pytest.raises(ValueError):
            st.misfit_static(t, t, t, _FakeTensor(torch.float64, (1,)))
    t = _FakeTensor(torch.float32)
    with pytest.raises(ValueError):
        st.misfit_static(t, t, t, _FakeTensor(torch.float64, (0,), n=0))
    with pytest.raises(ValueError):
        st.misfit_static(t, t, t, _FakeTensor(torch.float32, (1,)))


def simulate(kind, T, ops, wave):
    """Track which time level each buffer holds; check every read."""
    buf = {0: -1, 1: 0, 2: None, 3: None}
    t = 0
    for op, levels, in_p, in_c, out_p, out_c in ops:
        if op == 1:
            buf[out_c] = buf[in_c]
            continue
        assert buf[in_c] == t, (ops, t)
        if wave:
            assert buf[in_p] == t - 1
        assert out_c != in_c
        if levels >= 2:
            # a blocked pass reads neighbours of its inputs: it may not
            # overwrite them
            assert out_c not in (in_p, in_c) if wave else out_c != in_c
            if out_p >= 0:
                assert out_p not in (in_p, in_c)
        elif wave and out_c != in_p:
            assert out_c not in (in_p, in_c) and out_p not in (in_p, in_c)
        if out_p >= 0:
            buf[out_p] = t + levels - 1
        elif wave:
            buf[in_c] = t  # unchanged; the new prev is the old cur
        buf[out_c] = t + levels
        t += levels
    assert t == T
    return buf


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("b", [1, 2, 3, 4, 5, 8])
@pytest.mark.parametrize("dtype", [0, 1])
def test_schedule_leaves_state_in_caller_buffers(st, kind, b, dtype):
    wave = st.SECOND_ORDER[kind]
    for T in range(0, 40):
        ops = st.schedule(kind, T, b, dtype)
        buf = simulate(kind, T, ops, wave)
        if T > 0:
            assert buf[1] == T and buf[0] == T - 1, (kind, T, b, ops)
            npass = sum(1 for o in ops if o[0] == 0)
            ncopy = sum(1 for o in ops if o[0] == 1)
            # passes never exceed T; at most 2 copies (T = 1)
            assert npass <= T
            assert all(o[1] == 1 or o[1] <= b for o in ops if o[0] == 0)
            assert ncopy <= (2 if T == 1 else 1)
        else:
            assert ops == []


def _header_enum(prefix):
    src = open(os.path.join(ROOT, "include", "stencil.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return {m.group(1): int(m.group(2)) for m in re.finditer(r"\b" + prefix + r"([A-Z0-9_]+)\s*=\s*(-?\d+)", src)}


def test_binding_option_constants_match_header(st):
    """Every STENCIL_OPT_* value of the header is the binding's OPT_* constant
    of the same name (and the binding defines no other)."""
    hdr = _header_enum("STENCIL_OPT_")
    assert hdr and hdr == {k[4:]: v for k, v in vars(st).items() if k.startswith("OPT_")}


def test_binding_status_constants_match_header(st):
    hdr = _header_enum("STENCIL_")
    for name in ("OK", "EINVAL", "EUNSUPPORTED", "ENOMEM", "ECUDA", "ETIMEOUT"):
        assert getattr(st, name) == hdr[name], name


@pytest.mark.parametrize("levels", [1, 2])
@pytest.mark.parametrize("G", [1, 2, 3, 4, 7, 8, 16])
def test_adjoint_schedule_covers_steps_and_keeps_the_ring_safe(st, levels, G):
    """The adjoint's host program with gradient batches (stencil_adjoint_schedule),
    checked by simulating its two streams: every step is swept once, in
    order; a two-level sweep (levels = 2) never straddles a gradient batch
    and is used wherever two steps fit; each batch holds at most G steps and
    is waited for before the sweeps of the batch two later start; no sweep
    overwrites a ring slot that a gradient batch not yet waited for reads,
    and every sweep still finds its inputs (the two previous levels) in
    their slots."""
    NSL = 2 * G + 2
    for T in range(0, 41):
        ops = st.adjoint_schedule(T, G, levels)
        slot_level = {}          # ring slot -> level it holds
        done_upto = -1           # gradient batches known complete on the sweep stream
        issued = []              # gradient batches issued: (batch, levels read)
        pending = []             # steps swept since the last gradient batch
        next_step, next_batch = 1, 0
        for op, a, b in ops:
            if op == 0:          # wait for batch a - 2
                assert a >= 2 and a == next_batch and not pending
                done_upto = max(done_upto, a - 2)
            elif op == 1:        # sweep of steps a .. a+b-1
                assert a == next_step and b in ((1, 2) if levels == 2 else (1,))
                if levels == 2 and G >= 2 and len(pending) + 2 <= G and a + 1 <= T:
                    assert b == 2, "a pair fits"
                assert len(pending) + b <= G, "a sweep straddles a gradient batch"
                if len(pending) == 0 and next_batch >= 2:
                    assert done_upto >= next_batch - 2, "batch two back not waited for"
                for j in range(a, a + b):
                    for src in (j - 2, j - 1):          # inputs: levels in the ring or the caller's pair
                        if src >= 1:
                            assert slot_level.get((src - 1) % NSL) == src, "input overwritten"
                    slot = (j - 1) % NSL
                    for bb, reads in issued:
                        if bb > done_upto:
                            assert slot not in {(L - 1) % NSL for L in reads if L >= 1}, \
                                f"T={T}: step {j} overwrites a slot batch {bb} may still read"
                    slot_level[slot] = j
                    pending.append(j)
                next_step = a + b
            else:                # gradient batch a of b steps: reads level j-1 of each step j
                assert a == next_batch and b == len(pending) and 1 <= b <= G
                issued.append((a, [j - 1 for j in pending]))
                pending = []
                next_batch += 1
        assert next_step == T + 1 and not pending
        assert sum(k for op, _, k in ops if op == 2) == T


def test_adjoint_schedule_rejects_bad_arguments(st):
    for args in ((-1, 4, 1), (8, 0, 1), (8, 17, 1), (8, 4, 3)):
        with pytest.raises(st.StencilError):
            st.adjoint_schedule(*args)
