"""Helpers of the GPU parity tests: run the CUDA path through the C ABI on
seeded inputs and compare with the FP64 oracle."""
import numpy as np

F64, F32 = 0, 1
EPS32 = 2.0 ** -24


def torch_mod():
    import torch
    return torch


def to_dev(a, dtype):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float64 if dtype == F64 else torch.float32)


def to_np(t):
    return t.detach().to("cpu", dtype=torch_mod().float64).numpy()


def normwise_err(g, o):
    """max |g - o| / max |o| over all entries (the halo is zero in both)."""
    den = np.abs(o).max()
    return float(np.abs(g - o).max() / (den if den > 0 else 1.0))


def fp32_bound(kind, T, R):
    """Stated FP32 bound on the normwise error against the FP64 oracle:
    FP32 rounding of the inputs plus, per step, (number of terms + 2)
    roundings of size 2^-24; the wave kinds are not contractive in the
    max-norm, so their per-step growth factor is taken as T (linear growth
    of the leapfrog error), with a safety factor of 4."""
    terms = 6 * R + 3
    if kind in (3, 4, 6):
        return 4.0 * (T + 1) * (T + 1) * terms * EPS32
    return 4.0 * (T + 1) * terms * EPS32


def gpu_forward(plan_cls, wk, dtype, T=None, rcv_z=None, time_block=None, scheme=None, variant=None,
                expect_block=None):
    """Run stencil_forward on a workload; returns numpy (u_prev, u, trace).
    expect_block: the block depth the plan must report (the requested pass
    kernel serves the geometry)."""
    torch = torch_mod()
    T = wk.T if T is None else T
    nx, ny, nz = wk.n
    plan = plan_cls(wk.kind, nx, ny, nz, dtype)
    if time_block is not None:
        plan.set(1, time_block)
    if scheme is not None:
        plan.set(2, scheme)
    if variant is not None:
        plan.set(5, variant)
    if expect_block is not None:
        assert plan.get(1) == expect_block
    up = to_dev(wk.u_prev, dtype)
    u = to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    tr = None
    if rcv_z is not None:
        tr = torch.zeros((T, ny, nx), device="cuda", dtype=up.dtype)
    plan.forward(up, u, wk.w, W, T, trace=tr, rcv_z=rcv_z or 0)
    torch.cuda.synchronize()
    out = (to_np(up), to_np(u), to_np(tr) if tr is not None else None)
    plan.close()
    return out
