"""Measured error of the GPU sweeps against the FP64 oracle over all T steps,
per stencil, dtype and step count, in each plan's default launch
configuration (the one bench.py times).

* 512^3 at the full step counts of the benchmark configurations -- 7-point
  variable (T = 64), 25-point constant wave (T = 100), 25-point variable
  wave (T = 64) -- every entry of u^T compared: FP64 within 1e-12
  normwise, FP32 within the stated FP32 bar (4 x the error of the oracle's
  own FP32 evaluation of the same sweep).
* 128^3, every kind, seeds 0, 1 and 2: the same bars.

The normwise errors (max |g - o| / max |o| of u^T) of every case, and those
of the oracle's FP32 evaluation, are appended as JSON lines to the file named
by the environment variable STENCIL_ERROR_TABLE when it is set.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1410_3060_gb300 import workloads as wl
from gpu_util import F32, F64, fp32_bar, normwise_err, to_dev, to_np

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

T_OF = {wl.J7_CONST: 64, wl.J7_VAR: 64, wl.W25_CONST: 100, wl.W25_VAR: 64, wl.J25_VAR: 64, wl.W25_ALPHA: 64}


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def record(row):
    path = os.environ.get("STENCIL_ERROR_TABLE")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(row) + "\n")


def gpu_run(st, wk, dtype, T):
    import torch
    nx, ny, nz = wk.n
    plan = st.Plan(wk.kind, nx, ny, nz, dtype)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, T)
    plan.check()
    info = (plan.get(st.OPT_TIME_BLOCK), plan.get(st.OPT_SCHEME), plan.get(st.OPT_VARIANT))
    plan.close()
    out = to_np(u)
    del up, u, W
    torch.cuda.empty_cache()
    return out, info


def measure(st, wk, T, n, seed):
    threads = oracle.oracle.default_threads()
    _, o64, _ = oracle.forward(wk.kind, wk.u_prev, wk.u, wk.w, wk.W, T, threads=threads)
    _, o32, _ = oracle.forward_f32(wk.kind, wk.u_prev, wk.u, wk.w, wk.W, T, threads=threads)
    e32_oracle = normwise_err(o32, o64)
    for dtype in (F64, F32):
        g, (b, scheme, variant) = gpu_run(st, wk, dtype, T)
        err = normwise_err(g, o64)
        bar = 1e-12 if dtype == F64 else fp32_bar(o64, o32)
        record({"kind": wl.KIND_NAMES[wk.kind], "n": n, "T": T, "seed": seed,
                "dtype": "f64" if dtype == F64 else "f32", "normwise_err": err,
                "oracle_f32_err": e32_oracle, "bar": bar, "time_block": b, "scheme": scheme,
                "variant": variant})
        assert err <= bar, (wk.kind, dtype, err, bar, e32_oracle)


@pytest.mark.parametrize("kind", [wl.J7_VAR, wl.W25_CONST, wl.W25_VAR])
def test_full_steps_512(st, kind):
    n, T = 512, T_OF[kind]
    wk = wl.j7_var(n, T, seed=0) if kind == wl.J7_VAR else wl.make(kind, n, T, seed=0)
    measure(st, wk, T, n, 0)


@pytest.mark.parametrize("kind", [wl.J7_CONST, wl.J7_VAR, wl.W25_CONST, wl.W25_VAR, wl.J25_VAR, wl.W25_ALPHA])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_full_steps_128_seeds(st, kind, seed):
    n, T = 128, T_OF[kind]
    measure(st, wl.make(kind, n, T, seed=seed), T, n, seed)
