"""Temporally blocked adjoint (Sect. 4.1 wavefront applied to the
transposed sweep, two levels per pass: the register wavefront for the
7-point kinds, the two-level pass for the 13-array kinds) against the FP64
oracle's adjoint: both levels, residual injection on every level, the
coefficient gradient in batches that pair levels or not, ragged tiles in x,
y and z; plus the adjoint identity of the blocked adjoint with the forward."""
import numpy as np
import pytest

import oracle
from paper_1410_3060_gb300 import workloads as wl
from gpu_util import F32, F64, normwise_err, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def rand_interior(n, R, rng):
    a = np.zeros(wl.padded_shape(n, R))
    nx, ny, nz = n
    a[R:R + nz, R:R + ny, R:R + nx] = rng.uniform(-1, 1, size=(nz, ny, nx))
    return a


def run_case(st, kind, dtype, n, T, grad_batch, variant=0, seed=0, rz=None):
    import torch
    rng = np.random.default_rng(100 + 7 * kind + seed)
    wk = wl.make(kind, n, T, seed=seed)
    R = wk.R
    l2, l1 = rand_interior(n, R, rng), rand_interior(n, R, rng)
    states = np.stack([rand_interior(n, R, rng) for _ in range(T)])
    res = rng.uniform(-1, 1, size=(T, n[1], n[0]))
    rz = n[2] // 3 if rz is None else rz
    k = oracle.NUM_ARRAYS[kind]
    want_grad = k > 0 and grad_batch is not None
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == F32 else (lambda a: a)
    W = cast(wk.W) if wk.W is not None else None
    og = np.zeros((k,) + l1.shape) if want_grad else None
    ol2, ol1 = oracle.adjoint(kind, cast(l2), cast(l1), wk.w, W, T, states=cast(states), residual=cast(res),
                              rcv_z=rz, grad=og, threads=8)
    plan = st.Plan(kind, *n, dtype)
    if variant:
        plan.set(st.OPT_VARIANT, variant)
    plan.set(st.OPT_ADJ_TIME_BLOCK, 2)
    assert plan.get(st.OPT_ADJ_TIME_BLOCK) == 2
    if want_grad:
        plan.set(st.OPT_GRAD_BATCH, grad_batch)
    gl2, gl1 = to_dev(l2, dtype), to_dev(l1, dtype)
    gg = torch.zeros((k,) + l1.shape, device="cuda", dtype=torch.float64) if want_grad else None
    plan.adjoint(gl2, gl1, wk.w, to_dev(wk.W, dtype) if wk.W is not None else None, T,
                 fwd_states=[to_dev(s_, dtype) for s_ in states] if want_grad else None,
                 residual=to_dev(res, dtype), rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    plan.check()
    out = (to_np(gl2), to_np(gl1), to_np(gg) if want_grad else None)
    plan.close()
    return out, (ol2, ol1, og)


# (nx, ny, nz): several 64-column tiles with a ragged last one (nx + 2 a
# multiple of 4 and not), ragged y tiles, z chunks
SHAPES = [(130, 75, 70), (62, 37, 23), (200, 33, 18)]


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("T", [5, 8])
def test_blocked_adjoint_matches_oracle(st, kind, dtype, shape, T):
    """No gradient: every pass but a final one-level pass has two levels."""
    (g2, g1, _), (o2, o1, _) = run_case(st, kind, dtype, shape, T, None)
    tol = 1e-12 if dtype == F64 else 2e-5
    assert normwise_err(g1, o1) <= tol
    assert normwise_err(g2, o2) <= tol


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("grad_batch", [1, 2, 3, 8])
@pytest.mark.parametrize("T", [7, 9])
def test_blocked_adjoint_gradient(st, dtype, grad_batch, T):
    """With the coefficient gradient: levels are paired inside gradient
    batches (batch 1: no pairs; batch 3: a pair and a single level); the
    gradient sums lam^{n+1} d(A u^n)/dA over every level."""
    (g2, g1, gg), (o2, o1, og) = run_case(st, 2, dtype, (130, 45, 40), T, grad_batch)
    tol = 1e-12 if dtype == F64 else 2e-5
    assert normwise_err(g1, o1) <= tol
    assert normwise_err(g2, o2) <= tol
    assert normwise_err(gg, og) <= tol


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("variant", [10, 11, 12])
def test_blocked_adjoint_tiles(st, kind, variant):
    """Every register wavefront tile serves the depth-2 adjoint (FP64)."""
    (g2, g1, _), (o2, o1, _) = run_case(st, kind, F64, (150, 70, 40), 6, None, variant=variant)
    assert normwise_err(g1, o1) <= 1e-12
    assert normwise_err(g2, o2) <= 1e-12


@pytest.mark.parametrize("kind", [1, 2])
@pytest.mark.parametrize("rz", [0, 17])
def test_blocked_adjoint_receiver_at_chunk_edges(st, kind, rz):
    """Residual planes on the first plane and inside the lattice, in FP64, on
    a lattice tall enough for several z chunks."""
    (g2, g1, _), (o2, o1, _) = run_case(st, kind, F64, (62, 37, 150), 6, None, rz=rz)
    assert normwise_err(g1, o1) <= 1e-12
    assert normwise_err(g2, o2) <= 1e-12


@pytest.mark.parametrize("kind", [1, 2])
def test_blocked_adjoint_dot_product(st, kind):
    """<F_T b, y> = <b, F_T^T y> with the GPU forward and the blocked GPU
    adjoint (FP64, first-order kinds)."""
    import torch
    rng = np.random.default_rng(60 + kind)
    n, T = (70, 45, 33), 7
    wk = wl.make(kind, n, T, seed=9)
    R = wk.R
    b, x, y = (rand_interior(n, R, rng) for _ in range(3))
    plan = st.Plan(kind, *n, F64)
    W = to_dev(wk.W, F64) if wk.W is not None else None
    ga, gb = to_dev(np.zeros_like(b), F64), to_dev(b, F64)
    plan.forward(ga, gb, wk.w, W, T)
    plan.set(st.OPT_ADJ_TIME_BLOCK, 2)
    gx, gy = to_dev(x, F64), to_dev(y, F64)
    plan.adjoint(gx, gy, wk.w, W, T)
    torch.cuda.synchronize()
    lhs = np.sum(to_np(gb) * y)
    rhs = np.sum(b * to_np(gy))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    plan.close()


# the 13-array kinds in FP32 (the two-level pass's adjoint): nx a multiple of
# 4, several 64 x 16 tiles with ragged edges, z chunks
SHAPES25 = [(136, 45, 40), (64, 19, 30), (200, 33, 70)]


@pytest.mark.parametrize("kind", [4, 5])
@pytest.mark.parametrize("shape", SHAPES25)
@pytest.mark.parametrize("T", [5, 8])
def test_blocked_adjoint_25pt_matches_oracle(st, kind, shape, T):
    """The two-level adjoint pass of the 13-array kinds (FP32), no gradient."""
    (g2, g1, _), (o2, o1, _) = run_case(st, kind, F32, shape, T, None)
    assert normwise_err(g1, o1) <= 2e-5
    assert normwise_err(g2, o2) <= 2e-5


@pytest.mark.parametrize("kind", [4, 5])
@pytest.mark.parametrize("grad_batch", [1, 2, 3, 8])
def test_blocked_adjoint_25pt_gradient(st, kind, grad_batch):
    """With the FP64 coefficient gradient: levels paired inside gradient
    batches, against the oracle."""
    (g2, g1, gg), (o2, o1, og) = run_case(st, kind, F32, (136, 45, 40), 9, grad_batch)
    assert normwise_err(g1, o1) <= 2e-5
    assert normwise_err(g2, o2) <= 2e-5
    assert normwise_err(gg, og) <= 2e-5


def test_blocked_adjoint_option(st):
    """Depth 2 is served for the 7-point kinds and, in FP32, the 13-array
    kinds (default 1 for them); reading the option gives the depth the
    adjoint runs."""
    p = st.Plan(wl.W25_VAR, 32, 16, 16, F32)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 1
    p.set(st.OPT_ADJ_TIME_BLOCK, 2)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 2
    with pytest.raises(st.StencilError):
        p.set(st.OPT_ADJ_TIME_BLOCK, 3)
    p.close()
    for kind, dtype in ((wl.W25_VAR, F64), (wl.W25_CONST, F32), (wl.W25_ALPHA, F32)):
        p = st.Plan(kind, 32, 16, 16, dtype)
        with pytest.raises(st.StencilError):
            p.set(st.OPT_ADJ_TIME_BLOCK, 2)
        p.close()
    # default: depth 2 in FP32, 1 in FP64
    p = st.Plan(wl.J7_VAR, 32, 16, 16, F32)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 2
    p.set(st.OPT_ADJ_TIME_BLOCK, 1)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 1
    p.close()
    p = st.Plan(wl.J7_VAR, 32, 16, 16, F64)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 1
    p.set(st.OPT_ADJ_TIME_BLOCK, 2)
    assert p.get(st.OPT_ADJ_TIME_BLOCK) == 2
    p.close()
    # an odd padded row has no aligned vector layout: not served
    p = st.Plan(wl.J7_VAR, 33, 16, 16, F32)
    with pytest.raises(st.StencilError):
        p.set(st.OPT_ADJ_TIME_BLOCK, 2)
    p.close()


@pytest.mark.parametrize("kind,dtype,shape", [(2, F32, (66, 40, 30)), (2, F64, (66, 40, 30)),
                                              (4, F32, (64, 19, 30))])
def test_tune_adjoint_picks_a_depth_and_leaves_inputs(st, kind, dtype, shape):
    """tune.tune_adjoint times the served depths on copies: the caller's
    pair and gradient are untouched, the plan runs the chosen depth, and the
    adjoint it then computes matches the oracle."""
    import torch
    from paper_1410_3060_gb300 import tune
    rng = np.random.default_rng(90 + kind)
    T = 6
    wk = wl.make(kind, shape, T, seed=3)
    R = wk.R
    l2, l1 = rand_interior(shape, R, rng), rand_interior(shape, R, rng)
    states = np.stack([rand_interior(shape, R, rng) for _ in range(T)])
    res = rng.uniform(-1, 1, size=(T, shape[1], shape[0]))
    rz = shape[2] // 2
    k = oracle.NUM_ARRAYS[kind]
    cast = (lambda a: a.astype(np.float32).astype(np.float64)) if dtype == F32 else (lambda a: a)
    og = np.zeros((k,) + l1.shape)
    ol2, ol1 = oracle.adjoint(kind, cast(l2), cast(l1), wk.w, cast(wk.W), T, states=cast(states),
                              residual=cast(res), rcv_z=rz, grad=og, threads=8)
    plan = st.Plan(kind, *shape, dtype)
    plan.set(st.OPT_GRAD_BATCH, 4)
    gl2, gl1 = to_dev(l2, dtype), to_dev(l1, dtype)
    W = to_dev(wk.W, dtype)
    gs = [to_dev(s_, dtype) for s_ in states]
    gres = to_dev(res, dtype)
    gg = torch.zeros((k,) + l1.shape, device="cuda", dtype=torch.float64)
    out = tune.tune_adjoint(plan, gl2, gl1, wk.w, W, T, fwd_states=gs, residual=gres, rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    assert out["adjoint_levels_per_pass"] in (1, 2)
    assert plan.get(st.OPT_ADJ_TIME_BLOCK) == out["adjoint_levels_per_pass"]
    assert len(out["table"]) == (2 if (dtype == F32 or kind == 2) else 1)
    np.testing.assert_array_equal(to_np(gl1), cast(l1))
    np.testing.assert_array_equal(to_np(gl2), cast(l2))
    assert not to_np(gg).any()
    plan.adjoint(gl2, gl1, wk.w, W, T, fwd_states=gs, residual=gres, rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    tol = 1e-12 if dtype == F64 else 2e-5
    assert normwise_err(to_np(gl1), ol1) <= tol
    assert normwise_err(to_np(gl2), ol2) <= tol
    assert normwise_err(to_np(gg), og) <= tol
    plan.close()
