"""Parity of the temporally blocked passes (several time levels per sweep)
with the FP64 oracle: both y schemes (overlapped tiles; diamond split
tiling with edge bands), every kind, block depths, sizes spanning several
tiles in x, y and z with ragged tails, receiver traces of every level."""
import numpy as np
import pytest

import oracle
from paper_1410_3060_gb300 import workloads as wl
from gpu_util import F32, check_fp32, gpu_forward, normwise_err, oracle_both

pytestmark = pytest.mark.gpu

R1 = [1, 2]
R4 = [3, 4, 5, 6]


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def cases():
    out = []
    for kind in R1:
        for b in (2, 3, 4):
            for scheme in (1, 2):
                out.append((kind, b, scheme))
    for kind in R4:
        for scheme in (1, 2):
            out.append((kind, 2, scheme))
    return out


@pytest.mark.parametrize("kind,b,scheme", cases())
@pytest.mark.parametrize("shape", [(130, 75, 70), (41, 37, 23)])
@pytest.mark.parametrize("T", [9, 4])
def test_blocked_forward_fp32(st, kind, b, scheme, shape, T):
    wk = wl.make(kind, shape, T, seed=3)
    rz = shape[2] // 3
    o64, o32 = oracle_both(wk, T, rcv_z=rz)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F32, rcv_z=rz, time_block=b, scheme=scheme)
    check_fp32((gp, gu, gtr), o64, o32)
    R = wk.R
    halo = np.ones(gu.shape, bool)
    halo[R:-R, R:-R, R:-R] = False
    assert not gu[halo].any() and not gp[halo].any()


@pytest.mark.parametrize("kind,b,scheme", [(1, 4, 2), (2, 4, 1), (4, 2, 2), (3, 2, 1)])
def test_blocked_matches_plain_gpu(st, kind, b, scheme):
    """The blocked pass applies the same per-point update as the plain sweep:
    results agree to a few FP32 roundings per step."""
    shape = (96, 80, 64)
    T = 8
    wk = wl.make(kind, shape, T, seed=4)
    _, gu_b, _ = gpu_forward(st.Plan, wk, F32, time_block=b, scheme=scheme)
    _, gu_p, _ = gpu_forward(st.Plan, wk, F32, time_block=1)
    assert normwise_err(gu_b, gu_p) <= 8 * T * 2.0 ** -24 * (T if kind in (3, 4, 6) else 1)


@pytest.mark.parametrize("kind", R1)
@pytest.mark.parametrize("scheme", [1, 2])
@pytest.mark.parametrize("shape", [(70, 45, 40), (33, 19, 11)])
def test_blocked_forward_fp64(st, kind, scheme, shape):
    """FP64 two-level passes match the oracle to 1e-12."""
    from gpu_util import F64
    T = 7
    wk = wl.make(kind, shape, T, seed=9)
    rz = 3
    op, ou, otr = oracle.forward(kind, wk.u_prev, wk.u, wk.w, wk.W, T, rcv_z=rz, threads=8)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F64, rcv_z=rz, time_block=2, scheme=scheme)
    assert normwise_err(gu, ou) <= 1e-12
    assert normwise_err(gp, op) <= 1e-12
    assert normwise_err(gtr, otr) <= 1e-12


def test_time_block_option_roundtrip(st):
    p = st.Plan(1, 32, 32, 32, F32)
    assert p.get(2) == 3 and p.get(1) == 3 and p.get(5) == 12   # FP32 7-point defaults
    q = st.Plan(2, 32, 32, 32, F32)
    assert q.get(2) == 3 and q.get(1) == 2 and q.get(5) == 11
    q.close()
    p.set(2, 2)                                                  # shared-memory diamond tiles
    p.set(1, 4)
    assert p.get(1) == 4
    assert p.get(3) >= 3 * 34 * 34 * 34 * 4  # three band fields
    p.set(1, 1)
    assert p.get(1) == 1
    with pytest.raises(st.StencilError):
        p.set(1, 7)
    p.close()


# ---- register wavefront (scheme 3; tile variants 10-12 and, FP32 only,
# 17 -- 4 points per thread row -- also for one-level passes)

WF_SHAPES = [(130, 75, 70), (62, 37, 23), (200, 33, 18)]


@pytest.mark.parametrize("kind", R1)
@pytest.mark.parametrize("b", [1, 2, 3, 4])
@pytest.mark.parametrize("variant", [10, 11, 12, 17])
@pytest.mark.parametrize("shape", WF_SHAPES)
@pytest.mark.parametrize("T", [9, 4])
def test_wavefront_forward_fp32(st, kind, b, variant, shape, T):
    """Register wavefront passes of depth b (b = 1: every pass one level)
    against the oracle; the plan must run the requested depth."""
    wk = wl.make(kind, shape, T, seed=13)
    rz = shape[2] // 3
    o64, o32 = oracle_both(wk, T, rcv_z=rz)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F32, rcv_z=rz, time_block=b, scheme=3, variant=variant,
                              expect_block=b)
    check_fp32((gp, gu, gtr), o64, o32)
    R = wk.R
    halo = np.ones(gu.shape, bool)
    halo[R:-R, R:-R, R:-R] = False
    assert not gu[halo].any() and not gp[halo].any()


@pytest.mark.parametrize("kind", R1)
@pytest.mark.parametrize("b", [1, 2])
@pytest.mark.parametrize("variant", [10, 11, 12])
@pytest.mark.parametrize("shape", [(70, 45, 40), (34, 19, 11)])
def test_wavefront_forward_fp64(st, kind, b, variant, shape):
    """FP64 register wavefront passes match the oracle to 1e-12."""
    from gpu_util import F64
    T = 7
    wk = wl.make(kind, shape, T, seed=19)
    rz = 3
    op, ou, otr = oracle.forward(kind, wk.u_prev, wk.u, wk.w, wk.W, T, rcv_z=rz, threads=8)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F64, rcv_z=rz, time_block=b, scheme=3, variant=variant,
                              expect_block=b)
    assert normwise_err(gu, ou) <= 1e-12
    assert normwise_err(gp, op) <= 1e-12
    assert normwise_err(gtr, otr) <= 1e-12


@pytest.mark.parametrize("kind", R1)
def test_wavefront_matches_plain_gpu(st, kind):
    """Depth-4 register wavefront vs the plain sweep: a few FP32 roundings
    per step apart."""
    shape, T = (256, 96, 80), 8
    wk = wl.make(kind, shape, T, seed=21)
    _, gu_w, _ = gpu_forward(st.Plan, wk, F32, time_block=4, scheme=3, expect_block=4)
    _, gu_p, _ = gpu_forward(st.Plan, wk, F32, time_block=1)
    assert normwise_err(gu_w, gu_p) <= 8 * T * 2.0 ** -24


def test_wavefront_odd_row_falls_back(st):
    """An odd padded row length has no aligned vector layout: the plan runs
    plain passes (and still matches the oracle)."""
    shape, T = (41, 37, 23), 5
    wk = wl.make(1, shape, T, seed=2)
    o64, o32 = oracle_both(wk, T)
    _, gu, _ = gpu_forward(st.Plan, wk, F32, time_block=2, scheme=3, variant=10, expect_block=1)
    check_fp32((None, gu, None), o64, o32)


@pytest.mark.parametrize("kind,dtype", [(1, F32), (3, F32)])
def test_tune_forward_picks_a_valid_configuration(st, kind, dtype):
    """Run-time tuning times every candidate on copies of the caller's state,
    leaves the caller's state untouched, and the tuned plan still matches the
    oracle."""
    import torch
    from paper_1410_3060_gb300 import tune
    from gpu_util import to_dev, to_np
    shape, T = (80, 48, 40), 4
    wk = wl.make(kind, shape, T, seed=6)
    plan = st.Plan(kind, *shape, dtype)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    res = tune.tune_forward(plan, up, u, wk.w, W, T=T, reps=1)
    assert len(res["table"]) >= 10
    assert plan.get(1) == res["time_block"]
    np.testing.assert_array_equal(to_np(u), wk.u.astype(np.float32))   # caller's state untouched
    o64, o32 = oracle_both(wk, T)
    plan.forward(up, u, wk.w, W, T)
    plan.check()
    check_fp32((None, to_np(u), None), o64, o32)
    plan.close()


# ---- two-level pass of the 13-array 25-point kinds and the constant wave (scheme 4)

B25_SHAPES = [(136, 45, 40), (64, 19, 11), (200, 33, 70), (8, 7, 5)]


@pytest.mark.parametrize("kind", [3, 4, 5])
@pytest.mark.parametrize("shape", B25_SHAPES)
@pytest.mark.parametrize("T", [9, 4, 2])
def test_two_level_25pt_pass_fp32(st, kind, shape, T):
    """Scheme 4 at depth 2 against the oracle (FP32 bar): several tiles in x
    and y with ragged edges, z chunks, odd and even T (a plain pass for the
    remainder), receiver traces of both levels; the plan runs depth 2."""
    wk = wl.make(kind, shape, T, seed=23)
    rz = shape[2] // 2
    o64, o32 = oracle_both(wk, T, rcv_z=rz)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F32, rcv_z=rz, time_block=2, scheme=4, expect_block=2)
    check_fp32((gp, gu, gtr), o64, o32)
    R = wk.R
    halo = np.ones(gu.shape, bool)
    halo[R:-R, R:-R, R:-R] = False
    assert not gu[halo].any() and not gp[halo].any()


@pytest.mark.parametrize("kind", R1)
@pytest.mark.parametrize("dtype", [0, 1])
@pytest.mark.parametrize("T", [5, 6])
def test_forward_states_in_depth2_passes(st, kind, dtype, T):
    """stencil_forward_states on a plan of register wavefront passes: one
    depth-2 pass writes two consecutive states and the trace of both; every
    state and trace row against the oracle's steps (FP64 plans set scheme 3
    and depth 2 explicitly; FP32 plans run them by default)."""
    import torch
    from gpu_util import F64, to_dev, to_np
    shape = (130, 45, 40)
    wk = wl.make(kind, shape, T, seed=23)
    rz = 17
    plan = st.Plan(kind, *shape, dtype)
    if dtype == F64:
        plan.set(st.OPT_SCHEME, 3)
        plan.set(st.OPT_TIME_BLOCK, 2)
    assert plan.get(st.OPT_TIME_BLOCK) >= 2
    tdt = plan.torch_dtype()
    states = [torch.zeros(plan.padded_shape, device="cuda", dtype=tdt) for _ in range(T)]
    trace = torch.zeros((T, shape[1], shape[0]), device="cuda", dtype=tdt)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward_states(to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype), wk.w, W, states, trace=trace, rcv_z=rz)
    torch.cuda.synchronize()
    p, c = wk.u_prev, wk.u
    tol = 1e-12 if dtype == F64 else 1e-5
    for t in range(T):
        p, c, tr = oracle.forward(kind, p, c, wk.w, wk.W, 1, rcv_z=rz, threads=8)
        assert normwise_err(to_np(states[t]), c) <= tol, t
        assert normwise_err(to_np(trace[t]), tr[0]) <= tol, t
    plan.close()
