"""Differentiable path on the GPU: recompute with stored states, batched
FP64 gradients, the dot-product identity of the GPU forward/adjoint pair,
and the checkpointed autograd loss against the FP64 oracle gradient and
finite differences on the 48^3 copy of the differentiable wave workload."""
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


@pytest.mark.parametrize("kind", [2, 4])
@pytest.mark.parametrize("dtype", [F64, F32])
def test_forward_states(st, kind, dtype):
    import torch
    n, T = (45, 38, 30), 5
    wk = wl.make(kind, n, T, seed=6)
    plan = st.Plan(kind, *n, dtype)
    states = [torch.zeros(plan.padded_shape, device="cuda", dtype=plan.torch_dtype()) for _ in range(T)]  # zero halo
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    plan.forward_states(up, u, wk.w, to_dev(wk.W, dtype), states)
    torch.cuda.synchronize()
    p, c = wk.u_prev, wk.u
    tol = 1e-12 if dtype == F64 else 1e-5
    for t in range(T):
        p, c, _ = oracle.forward(kind, p, c, wk.w, wk.W, 1)
        assert normwise_err(to_np(states[t]), c) <= tol
    np.testing.assert_array_equal(to_np(u), wk.u.astype(np.float32) if dtype == F32 else wk.u)
    plan.close()


@pytest.mark.parametrize("kind", [2, 4, 5, 6])
@pytest.mark.parametrize("batch", [3, 8])
@pytest.mark.parametrize("nx", [37, 40])
def test_batched_gradient_matches_oracle(st, kind, batch, nx):
    """Gradient batches of 3 and 8 steps over 9 steps; nx = 40 gives the
    13-array kinds the shared-memory tiled gradient kernel for batches of 8
    steps (the rest: one thread per point and axis)."""
    import torch
    rng = np.random.default_rng(20 + kind)
    n, T, rz = (nx, 29, 21), 9, 6
    wk = wl.make(kind, n, T, seed=5)
    R = wk.R
    l2, l1 = rand_interior(n, R, rng), rand_interior(n, R, rng)
    states = np.stack([rand_interior(n, R, rng) for _ in range(T)])
    res = rng.uniform(-1, 1, size=(T, n[1], n[0]))
    og = np.zeros((oracle.NUM_ARRAYS[kind],) + l1.shape)
    ol2, ol1 = oracle.adjoint(kind, l2, l1, wk.w, wk.W, T, states=states, residual=res, rcv_z=rz, grad=og)
    plan = st.Plan(kind, *n, F64)
    plan.set(st.OPT_GRAD_BATCH, batch)
    gl2, gl1 = to_dev(l2, F64), to_dev(l1, F64)
    gg = torch.zeros(og.shape, device="cuda", dtype=torch.float64)
    plan.adjoint(gl2, gl1, wk.w, to_dev(wk.W, F64), T, fwd_states=[to_dev(s, F64) for s in states],
                 residual=to_dev(res, F64), rcv_z=rz, grad=gg)
    torch.cuda.synchronize()
    assert normwise_err(to_np(gl1), ol1) <= 1e-12
    assert normwise_err(to_np(gl2), ol2) <= 1e-12
    assert normwise_err(to_np(gg), og) <= 1e-12
    plan.close()


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5, 6])
def test_gpu_dot_product(st, kind):
    """<F_T(a, b), (x, y)> = <(a, b), F_T^T (x, y)> with the GPU forward and
    adjoint (FP64), as in the oracle pin."""
    import torch
    rng = np.random.default_rng(30 + kind)
    n, T = (40, 33, 27), 6
    wk = wl.make(kind, n, T, seed=7)
    R = wk.R
    a, b, x, y = (rand_interior(n, R, rng) for _ in range(4))
    plan = st.Plan(kind, *n, F64)
    W = to_dev(wk.W, F64) if wk.W is not None else None
    ga, gb = to_dev(a, F64), to_dev(b, F64)
    plan.forward(ga, gb, wk.w, W, T)
    if st.SECOND_ORDER[kind]:
        gx, gy = to_dev(-x, F64), to_dev(y, F64)
        plan.adjoint(gx, gy, wk.w, W, T)
        torch.cuda.synchronize()
        lhs = np.sum(to_np(ga) * x) + np.sum(to_np(gb) * y)
        rhs = np.sum(a * -to_np(gx)) + np.sum(b * to_np(gy))
    else:
        gx, gy = to_dev(x, F64), to_dev(y, F64)
        plan.adjoint(gx, gy, wk.w, W, T)
        torch.cuda.synchronize()
        lhs = np.sum(to_np(gb) * y)
        rhs = np.sum(b * to_np(gy))
    assert abs(lhs - rhs) <= 1e-12 * max(1.0, abs(lhs))
    plan.close()


@pytest.fixture(scope="module")
def fwi48():
    fw = wl.fwi(48, T=60, K=10, seed=0)
    _, _, d = oracle.forward(wl.W25_VAR, fw.u0, fw.u0, None, fw.W_true, fw.T, rcv_z=fw.rcv_z, threads=8)
    loss, du0, dW = oracle.loss_and_gradient(wl.W25_VAR, fw.u0, fw.W, d, fw.T, fw.rcv_z, threads=8)
    return fw, d, loss, du0, dW


@pytest.mark.parametrize("dtype", [F64, F32])
def test_autograd_matches_oracle_gradient(st, fwi48, dtype):
    import torch
    from paper_1410_3060_gb300.autograd import MisfitRunner
    fw, d, oloss, odu0, odW = fwi48
    run = MisfitRunner(wl.W25_VAR, fw.n, fw.T, fw.K, fw.rcv_z, dtype=dtype)
    u0 = to_dev(fw.u0, dtype).requires_grad_(True)
    W = to_dev(fw.W, dtype).requires_grad_(True)
    loss = run(u0, W, to_dev(d, dtype))
    loss.backward()
    torch.cuda.synchronize()
    tol = 1e-10 if dtype == F64 else 2e-3
    assert abs(loss.item() - oloss) <= tol * oloss
    assert normwise_err(to_np(u0.grad), odu0) <= tol
    for k in range(13):
        assert normwise_err(to_np(W.grad[k]), odW[k]) <= tol, k
    run.close()


def test_autograd_finite_differences_gpu(st, fwi48):
    """Central differences of the GPU loss (FP64) along random directions."""
    import torch
    from paper_1410_3060_gb300.autograd import MisfitRunner
    fw, d, _, _, _ = fwi48
    run = MisfitRunner(wl.W25_VAR, fw.n, fw.T, fw.K, fw.rcv_z, dtype=F64)
    u0 = to_dev(fw.u0, F64).requires_grad_(True)
    W = to_dev(fw.W, F64).requires_grad_(True)
    dd = to_dev(d, F64)
    loss = run(u0, W, dd)
    loss.backward()
    rng = np.random.default_rng(3)
    R = 4
    du = to_dev(rand_interior(fw.n, R, rng), F64)
    h = 1e-3
    with torch.no_grad():
        fd = (run(u0 + h * du, W, dd).item() - run(u0 - h * du, W, dd).item()) / (2 * h)
    an = float((u0.grad * du).sum())
    assert abs(fd - an) <= 1e-6 * abs(an)
    for k in (0, 7):
        dw = torch.zeros_like(W)
        dw[k] = to_dev(rand_interior(fw.n, R, rng), F64) * float(W[k].detach().abs().max())
        h = 1e-6
        with torch.no_grad():
            fd = (run(u0, W + h * dw, dd).item() - run(u0, W - h * dw, dd).item()) / (2 * h)
        an = float((W.grad * dw).sum())
        assert abs(fd - an) <= 1e-5 * max(abs(an), abs(fd)), (k, fd, an)
    run.close()


@pytest.mark.parametrize("overlap", [True, False])
def test_backward_pass_repeated(st, fwi48, overlap):
    """The forward pass keeps the last segment's states for the backward
    pass; a second backward pass on the same forward state recomputes them
    and gives the same gradients (both runner modes), which match the
    oracle's."""
    import torch
    from paper_1410_3060_gb300.autograd import MisfitRunner
    fw, d, _, odu0, odW = fwi48
    run = MisfitRunner(wl.W25_VAR, fw.n, fw.T, fw.K, fw.rcv_z, dtype=F64, overlap=overlap)
    u0, W, dd = to_dev(fw.u0, F64), to_dev(fw.W, F64), to_dev(d, F64)
    one = torch.ones((), dtype=torch.float64)
    _, state = run.forward_pass(u0, W, dd)
    du0a, dWa = run.backward_pass(state, W, one)
    du0a, dWa = du0a.clone(), dWa.clone()
    du0b, dWb = run.backward_pass(state, W, one)
    torch.cuda.synchronize()
    assert torch.equal(du0a, du0b) and torch.equal(dWa, dWb)
    assert normwise_err(to_np(du0a), odu0) <= 1e-10
    for k in range(13):
        assert normwise_err(to_np(dWa[k]), odW[k]) <= 1e-10, k
    run.close()


@pytest.mark.parametrize("dtype", [F64, F32])
def test_two_losses_summed_one_backward(st, fwi48, dtype):
    """Two losses of one runner built before a single backward(): each forward
    pass keeps its own checkpoints and residual, so the gradient of the sum
    is the sum of the oracle gradients (the second data set is the first
    scaled by 0.5, so its loss and gradient differ)."""
    import torch
    from paper_1410_3060_gb300.autograd import MisfitRunner
    fw, d, oloss, odu0, odW = fwi48
    d2 = 0.5 * d
    oloss2, odu02, odW2 = oracle.loss_and_gradient(wl.W25_VAR, fw.u0, fw.W, d2, fw.T, fw.rcv_z, threads=8)
    run = MisfitRunner(wl.W25_VAR, fw.n, fw.T, fw.K, fw.rcv_z, dtype=dtype)
    u0 = to_dev(fw.u0, dtype).requires_grad_(True)
    W = to_dev(fw.W, dtype).requires_grad_(True)
    l1 = run(u0, W, to_dev(d, dtype))
    l2 = run(u0, W, to_dev(d2, dtype))
    (l1 + 3.0 * l2).backward()
    torch.cuda.synchronize()
    tol = 1e-10 if dtype == F64 else 2e-3
    assert abs(l1.item() - oloss) <= tol * oloss and abs(l2.item() - oloss2) <= tol * oloss2
    assert normwise_err(to_np(u0.grad), odu0 + 3.0 * odu02) <= tol
    for k in range(13):
        assert normwise_err(to_np(W.grad[k]), odW[k] + 3.0 * odW2[k]) <= tol, k
    assert len(run._pool) == 2     # both buffer sets returned after backward
    run.close()
