"""Parity of the CUDA path (through the C ABI) with the FP64 oracle on seeded
inputs: every kind, FP64 (normwise <= 1e-12) and FP32 (stated bound), sizes
spanning several tiles in x, y and z with ragged tails, T odd and even,
receiver traces, the adjoint, coefficient gradients and the misfit."""
import numpy as np
import pytest

import oracle
from paper_1410_3060_gb300 import workloads as wl
from gpu_util import F32, F64, check_fp32, gpu_forward, normwise_err, oracle_both, to_dev, to_np

pytestmark = pytest.mark.gpu

KINDS = [1, 2, 3, 4, 5, 6]
SHAPES = [(70, 45, 40), (33, 17, 9)]


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def oracle_forward(wk, T, rcv_z=None):
    return oracle.forward(wk.kind, wk.u_prev, wk.u, wk.w, wk.W, T, rcv_z=rcv_z, threads=8)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T", [1, 2, 5])
def test_forward_fp64(st, kind, shape, T):
    wk = wl.make(kind, shape, T, seed=1)
    rz = shape[2] // 2
    op, ou, otr = oracle_forward(wk, T, rcv_z=rz)
    gp, gu, gtr = gpu_forward(st.Plan, wk, F64, rcv_z=rz)
    assert normwise_err(gu, ou) <= 1e-12
    assert normwise_err(gp, op) <= 1e-12
    assert normwise_err(gtr, otr) <= 1e-12
    R = wk.R
    halo = np.ones(gu.shape, bool)
    halo[R:-R, R:-R, R:-R] = False
    assert not gu[halo].any() and not gp[halo].any()


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("T", [3, 8])
def test_forward_fp32(st, kind, T):
    shape = (70, 45, 40)
    wk = wl.make(kind, shape, T, seed=2)
    o64, o32 = oracle_both(wk, T)
    gp, gu, _ = gpu_forward(st.Plan, wk, F32)
    check_fp32((gp, gu), o64, o32)


def test_config_64cube_j7_const_fp64(st):
    """7-point constant, 64^3, zero Dirichlet halo, T = 8, FP64: every entry."""
    wk = wl.j7_const(64, 8, seed=0)
    op, ou, _ = oracle_forward(wk, 8)
    gp, gu, _ = gpu_forward(st.Plan, wk, F64)
    assert normwise_err(gu, ou) <= 1e-12
    assert normwise_err(gp, op) <= 1e-12


def test_zero_steps_leave_state(st):
    wk = wl.make(4, (20, 20, 20), 0, seed=3)
    gp, gu, _ = gpu_forward(st.Plan, wk, F64, T=0)
    np.testing.assert_array_equal(gu, wk.u)
    np.testing.assert_array_equal(gp, wk.u_prev)


def rand_interior(n, R, rng):
    a = np.zeros(wl.padded_shape(n, R))
    nx, ny, nz = n
    a[R:R + nz, R:R + ny, R:R + nx] = rng.uniform(-1, 1, size=(nz, ny, nx))
    return a


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("variant", [0, 5, 13, 15])
def test_adjoint_with_residual_and_gradient(st, kind, dtype, variant):
    """Adjoint sweeps (variant 13: the vectorised 25-point sweep serves the
    self-adjoint constant kind; other kinds keep their adjoint kernels)."""
    import torch
    rng = np.random.default_rng(10 + kind)
    n = (37, 29, 21) if variant < 13 else (40, 29, 21)
    T = 4
    wk = wl.make(kind, n, T, seed=4)
    R = wk.R
    l2 = rand_interior(n, R, rng)
    l1 = rand_interior(n, R, rng)
    states = np.stack([rand_interior(n, R, rng) for _ in range(T)])
    res = rng.uniform(-1, 1, size=(T, n[1], n[0]))
    rz = 7
    k = oracle.NUM_ARRAYS[kind]
    og = np.zeros((k,) + l1.shape) if k else None
    # cast inputs through the GPU dtype so both sides see the same values
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == F32 else (lambda a: a)
    W = cast(wk.W) if wk.W is not None else None
    ol2, ol1 = oracle.adjoint(kind, cast(l2), cast(l1), wk.w, W, T, states=cast(states), residual=cast(res),
                              rcv_z=rz, grad=og, threads=8)
    plan = st.Plan(kind, *n, dtype)
    plan.set(st.OPT_VARIANT, variant)
    gl2, gl1 = to_dev(l2, dtype), to_dev(l1, dtype)
    gst = [to_dev(s, dtype) for s in states]
    gg = torch.zeros((k,) + l1.shape, device="cuda", dtype=torch.float64) if k else None
    plan.adjoint(gl2, gl1, wk.w, to_dev(wk.W, dtype) if wk.W is not None else None, T,
                 fwd_states=gst if k else None, residual=to_dev(res, dtype), rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == F64 else 2e-5
    assert normwise_err(to_np(gl1), ol1) <= tol
    assert normwise_err(to_np(gl2), ol2) <= tol
    if k:
        assert normwise_err(to_np(gg), og) <= (1e-12 if dtype == F64 else 2e-5)
    plan.close()


@pytest.mark.parametrize("kind", [4, 5])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_adjoint_tiles_and_chunks(st, kind, dtype):
    """The default adjoint of the 13-array kinds (TMA-staged coefficients)
    over several x tiles (the last one ragged), ragged y tiles and several z
    chunks (the last one shorter), with the gradient in a batch of 8 steps
    (the shared-memory tiled kernel) and one of 1; against the oracle."""
    import torch
    rng = np.random.default_rng(40 + kind)
    n = (264, 40, 70)
    T = 9
    wk = wl.make(kind, n, T, seed=5)
    R = wk.R
    l2, l1 = rand_interior(n, R, rng), rand_interior(n, R, rng)
    states = np.stack([rand_interior(n, R, rng) for _ in range(T)])
    res = rng.uniform(-1, 1, size=(T, n[1], n[0]))
    rz = 33
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == F32 else (lambda a: a)
    og = np.zeros((13,) + l1.shape)
    ol2, ol1 = oracle.adjoint(kind, cast(l2), cast(l1), wk.w, cast(wk.W), T, states=cast(states),
                              residual=cast(res), rcv_z=rz, grad=og, threads=8)
    plan = st.Plan(kind, *n, dtype)
    assert plan.get(st.OPT_VARIANT) == 16
    plan.set(st.OPT_GRAD_BATCH, 8)
    gl2, gl1 = to_dev(l2, dtype), to_dev(l1, dtype)
    gg = torch.zeros((13,) + l1.shape, device="cuda", dtype=torch.float64)
    plan.adjoint(gl2, gl1, wk.w, to_dev(wk.W, dtype), T, fwd_states=[to_dev(s_, dtype) for s_ in states],
                 residual=to_dev(res, dtype), rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == F64 else 2e-5
    assert normwise_err(to_np(gl1), ol1) <= tol
    assert normwise_err(to_np(gl2), ol2) <= tol
    assert normwise_err(to_np(gg), og) <= tol
    assert st.wait_timeouts() == 0
    plan.close()


@pytest.mark.parametrize("dtype", [F64, F32])
def test_misfit(st, dtype):
    import torch
    rng = np.random.default_rng(5)
    T, ny, nx = 7, 13, 19
    tr = rng.uniform(-1, 1, size=(T, ny, nx))
    d = rng.uniform(-1, 1, size=(T, ny, nx))
    plan = st.Plan(4, nx, ny, 9, dtype)
    gtr, gd = to_dev(tr, dtype), to_dev(d, dtype)
    res = torch.empty_like(gtr)
    loss = torch.zeros(1, device="cuda", dtype=torch.float64)
    plan.misfit(gtr, gd, res, loss)
    torch.cuda.synchronize()
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == F32 else (lambda a: a)
    ol, orr = oracle.receiver_loss(cast(tr), cast(d))
    assert abs(loss.item() - ol) <= (1e-13 if dtype == F64 else 1e-6) * ol
    assert normwise_err(to_np(res), orr) <= (1e-15 if dtype == F64 else 1e-7)
    plan.close()


def test_bad_arguments_rejected(st):
    import torch
    plan = st.Plan(1, 16, 16, 16, F64)
    u = torch.zeros(plan.padded_shape, device="cuda", dtype=torch.float64)
    with pytest.raises(st.StencilError):
        plan.forward(u, u, [0.4, 0.1], None, 2)          # aliased pair
    v = torch.zeros(plan.padded_shape, device="cuda", dtype=torch.float64)
    with pytest.raises(st.StencilError):
        plan.forward(u, v, [0.4], None, 2)               # wrong weight count
    with pytest.raises(st.StencilError):
        plan.forward(u, v, [0.4, 0.1], None, -1)         # negative T
    tr = torch.zeros((2, 16, 16), device="cuda", dtype=torch.float64)
    with pytest.raises(st.StencilError):
        plan.forward(u, v, [0.4, 0.1], None, 2, trace=tr, rcv_z=16)  # receiver outside
    plan.close()


def test_fma_peak_probe(st):
    f64, clk = st.fma_peak(0)
    f32, _ = st.fma_peak(1)
    assert f64 > 1e11 and f32 > 1e13 and clk > 5e8


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("variant", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12, 13, 14, 15, 16])
def test_forward_tile_variants(st, kind, dtype, variant):
    """Every forward tile variant against the oracle (ragged tiles in x, y, z)."""
    check_forward_variant(st, kind, dtype, variant, (150, 45, 40))


@pytest.mark.parametrize("kind", [3, 4, 5, 6])
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("variant", [13, 14, 15, 16])
@pytest.mark.parametrize("shape", [(136, 45, 40), (64, 19, 11), (264, 9, 30)])
def test_vectorised_25pt_sweep(st, kind, dtype, variant, shape):
    """The vectorised 25-point sweep (nx a multiple of the vector width;
    variants 15, 16 staged by TMA) against the oracle: ragged tiles in x, y
    and z, receiver trace; no bounded wait gave up."""
    check_forward_variant(st, kind, dtype, variant, shape)


@pytest.mark.parametrize("kind", KINDS)
@pytest.mark.parametrize("variant", [17])
def test_forward_tile_variants_fp32_wide(st, kind, variant):
    """The FP32-only wavefront tile of 4 points per thread row (the other
    kinds run their default sweep) against the oracle; an FP64 plan
    rejects it."""
    check_forward_variant(st, kind, F32, variant, (150, 45, 40))
    plan = st.Plan(kind, 16, 16, 16, F64)
    with pytest.raises(st.StencilError):
        plan.set(st.OPT_VARIANT, variant)
    plan.close()


def check_forward_variant(st, kind, dtype, variant, shape):
    T = 3
    wk = wl.make(kind, shape, T, seed=8)
    rz = min(11, shape[2] - 1)
    o64, o32 = oracle_both(wk, T, rcv_z=rz)
    op, ou, otr = o64
    import gpu_util
    torch = gpu_util.torch_mod()
    nx, ny, nz = shape
    plan = st.Plan(kind, nx, ny, nz, dtype)
    plan.set(st.OPT_VARIANT, variant)
    assert plan.get(st.OPT_VARIANT) == variant
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    tr = torch.zeros((T, ny, nx), device="cuda", dtype=up.dtype)
    plan.forward(up, u, wk.w, to_dev(wk.W, dtype) if wk.W is not None else None, T, trace=tr, rcv_z=rz)
    plan.check()   # no bounded device wait gave up
    if dtype == F64:
        assert normwise_err(to_np(u), ou) <= 1e-12
        assert normwise_err(to_np(up), op) <= 1e-12
        assert normwise_err(to_np(tr), otr) <= 1e-12
    else:
        check_fp32((to_np(up), to_np(u), to_np(tr)), o64, o32)
    plan.close()


@pytest.mark.parametrize("kind,dtype", [(1, F32), (2, F64), (3, F32), (4, F32)])
def test_graph_replay_matches_direct(st, kind, dtype):
    """STENCIL_OPT_GRAPH: the captured pass program replayed on the caller's
    stream gives the same bits as direct launches, on a replay with the same
    arguments and after a new argument set (recapture)."""
    import gpu_util
    torch = gpu_util.torch_mod()
    shape, T = (64, 40, 30), 7
    wk = wl.make(kind, shape, T, seed=12)
    nx, ny, nz = shape
    W = to_dev(wk.W, dtype) if wk.W is not None else None

    def run(graph, reps):
        plan = st.Plan(kind, nx, ny, nz, dtype)
        plan.set(st.OPT_GRAPH, graph)
        assert plan.get(st.OPT_GRAPH) == graph
        outs = []
        for rep in range(reps):
            up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
            tr = torch.zeros((T, ny, nx), device="cuda", dtype=up.dtype)
            plan.forward(up, u, wk.w, W, T, trace=tr, rcv_z=5)
            if rep == 0:
                # same arguments again: a replay continues from the new state
                plan.forward(up, u, wk.w, W, T, trace=tr, rcv_z=5)
            torch.cuda.synchronize()
            outs.append((to_np(up), to_np(u), to_np(tr)))
        plan.close()
        return outs

    direct = run(0, 2)
    graph = run(1, 2)
    for d, g_ in zip(direct, graph):
        for a, b in zip(d, g_):
            np.testing.assert_array_equal(a, b)
