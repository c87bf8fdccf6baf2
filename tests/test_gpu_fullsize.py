"""Parity at the benchmark sizes (512^3), in the launch configuration
bench.py times (each plan's default passes), on sampled outputs.

The oracle cannot run a whole 512^3 time loop inside a test, so:

* 7-point kinds: u^T at a point depends only on the initial data inside the
  cube of half-width R T around it (the dependency cone of T steps).  The
  oracle runs the T steps on that cube; the cube's own halo, R T + 1 or more
  points from the sample, holds fixed values that cannot reach the sample in
  T steps, and where the cube meets the domain boundary the halo is the zero
  Dirichlet halo itself.  Every sampled GPU value of u^T (after all the
  blocked passes of the default program) must match to the dtype's bar.
* 25-point kinds (the cone of T = 64-100 steps covers the whole domain):
  one-step consistency at sampled points -- the GPU's last step recomputed
  by the oracle from the GPU's own (u^{T-2}, u^{T-1}) on the (2R+1)^3
  neighbourhood of each sample.
"""
import numpy as np
import pytest

import oracle
from paper_1410_3060_gb300 import workloads as wl
from gpu_util import F32, F64, EPS32, fp32_bar, to_dev

pytestmark = pytest.mark.gpu

N = 512


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def samples(n, seed):
    """Interior points (x, y, z): corners, edge and face points, the centre
    and seeded random points."""
    rng = np.random.default_rng(seed)
    pts = [(0, 0, 0), (n - 1, n - 1, n - 1), (0, n // 2, n - 1), (n - 1, 0, n // 3), (n // 2, n // 2, n // 2)]
    pts += [tuple(int(v) for v in rng.integers(0, n, 3)) for _ in range(3)]
    return pts


_cache = {}


def workload(kind, T):
    """The bench's 512^3 workload; the last one is kept (tests of one kind
    run consecutively, so each is generated once)."""
    key = (kind, T)
    if key not in _cache:
        _cache.clear()
        _cache[key] = wl.j7_var(N, T, seed=0) if kind == wl.J7_VAR else wl.make(kind, N, T, seed=0)
    return _cache[key]


def gpu_state(st, kind, dtype, wk, T):
    """Run the plan's default program for T steps; returns the device pair."""
    import torch
    plan = st.Plan(kind, N, N, N, dtype)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, T)
    torch.cuda.synchronize()
    plan.close()
    return up, u, W


@pytest.mark.parametrize("kind,dtype", [(wl.J7_VAR, F64), (wl.J7_VAR, F32), (wl.J7_CONST, F32)])
def test_dependency_cone_samples_512(st, kind, dtype):
    T = 64
    wk = workload(kind, T)
    R = wk.R
    _, u, W = gpu_state(st, kind, dtype, wk, T)
    for (x, y, z) in samples(N, 7):
        lo = [max(c - R * T, 0) for c in (x, y, z)]
        hi = [min(c + R * T, N - 1) for c in (x, y, z)]
        # padded slice of the cube plus its halo
        sl = (slice(lo[2], hi[2] + 1 + 2 * R), slice(lo[1], hi[1] + 1 + 2 * R), slice(lo[0], hi[0] + 1 + 2 * R))
        Wb = wk.W[(slice(None),) + sl] if wk.W is not None else None
        _, ob, _ = oracle.forward(kind, wk.u_prev[sl], wk.u[sl], wk.w, Wb, T, threads=8)
        if dtype == F64:
            tol = 1e-12
        else:
            # the FP32 bar of this cube: 4 x the error of the oracle's FP32 evaluation
            _, fb, _ = oracle.forward_f32(kind, wk.u_prev[sl], wk.u[sl], wk.w, Wb, T, threads=8)
            tol = fp32_bar(ob, fb)
        o = ob[z - lo[2] + R, y - lo[1] + R, x - lo[0] + R]
        g = float(u[z + R, y + R, x + R].item())
        scale = max(np.abs(ob).max(), 1e-300)
        assert abs(g - o) <= tol * scale, ((x, y, z), g, o, scale)


@pytest.mark.parametrize("dtype", [F64, F32])
@pytest.mark.parametrize("kind,T", [(wl.W25_CONST, 100), (wl.W25_VAR, 64)])
def test_last_step_samples_512(st, kind, T, dtype):
    import torch
    wk = workload(kind, T)
    R = wk.R
    plan = st.Plan(kind, N, N, N, dtype)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, T - 1)
    torch.cuda.synchronize()
    pts = samples(N, 11)
    # the (2R+1)^3 neighbourhoods of (u^{T-2}, u^{T-1}) the last step reads
    boxes = []
    for (x, y, z) in pts:
        sl = (slice(z, z + 2 * R + 1), slice(y, y + 2 * R + 1), slice(x, x + 2 * R + 1))
        boxes.append((up[sl].double().cpu().numpy(), u[sl].double().cpu().numpy(),
                      W[(slice(None),) + sl].double().cpu().numpy() if W is not None else None))
    plan.forward(up, u, wk.w, W, 1)
    torch.cuda.synchronize()
    plan.close()
    for (x, y, z), (bp, bu, bW) in zip(pts, boxes):
        _, ob, _ = oracle.forward(kind, bp, bu, wk.w, bW, 1)
        o = ob[R, R, R]
        g = float(u[z + R, y + R, x + R].item())
        scale = max(np.abs(bu).max(), np.abs(bp).max(), 1e-300)
        tol = 1e-13 if dtype == F64 else 16 * (6 * R + 3) * EPS32
        assert abs(g - o) <= tol * scale, ((x, y, z), g, o, scale)
