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


def fp32_bar(o64, o32):
    """Stated FP32 bar on the normwise error against the FP64 oracle: 4 times
    the normwise error of the oracle's own FP32 evaluation of the same sweep
    (oracle.forward_f32: the same FP32-rounded inputs, every update in FP32),
    with a floor of 4 FP32 ulps.  The bar scales with the real rounding
    error of the case (kind, T, size, data), not with a worst case."""
    return 4.0 * max(normwise_err(o32, o64), 4 * EPS32)


def oracle_both(wk, T=None, rcv_z=None, threads=8):
    """(FP64 oracle, its FP32 evaluation) of a workload: two triples
    (u_prev, u, trace)."""
    import oracle
    T = wk.T if T is None else T
    o64 = oracle.forward(wk.kind, wk.u_prev, wk.u, wk.w, wk.W, T, rcv_z=rcv_z, threads=threads)
    o32 = oracle.forward_f32(wk.kind, wk.u_prev, wk.u, wk.w, wk.W, T, rcv_z=rcv_z, threads=threads)
    return o64, o32


def check_fp32(g, o64, o32):
    """Every array of the GPU triple within the FP32 bar of its oracle pair
    (None entries skipped); returns the normwise errors."""
    errs = []
    for gi, oi, fi in zip(g, o64, o32):
        if gi is None or oi is None:
            continue
        e = normwise_err(gi, oi)
        assert e <= fp32_bar(oi, fi), (e, fp32_bar(oi, fi), normwise_err(fi, oi))
        errs.append(e)
    return errs


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
    plan.check()   # no bounded device wait gave up
    out = (to_np(up), to_np(u), to_np(tr) if tr is not None else None)
    plan.close()
    return out
