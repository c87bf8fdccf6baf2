"""The bounded plane waits of the TMA-staged sweeps give up cleanly.

A plan's test hook (STENCIL_OPT_TEST_SKIP_COPY) makes the first CTA of every
TMA-staged sweep skip issuing the copies of one plane, so that CTA waits for
a copy that never comes -- a wait nothing completes, with no copy in
flight for it.  With a short poll limit (STENCIL_OPT_WAIT_LIMIT) the wait
gives up: the whole CTA leaves its plane loop together, its issuing thread
waits for the copies it still has in flight, one timeout is counted, and
stencil_check reports STENCIL_ETIMEOUT.  The context stays usable: the same
plan without the hook then matches the oracle and checks clean.
"""
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


@pytest.mark.parametrize("dtype", [F32, F64])
@pytest.mark.parametrize("kind", [wl.W25_VAR, wl.W25_CONST])
def test_forward_wait_gives_up_with_etimeout(st, kind, dtype):
    import torch
    shape, T = (64, 24, 20), 3
    wk = wl.make(kind, shape, T, seed=5)
    plan = st.Plan(kind, *shape, dtype)
    plan.set(st.OPT_VARIANT, 16)
    plan.set(st.OPT_WAIT_LIMIT, 2000)
    plan.set(st.OPT_TEST_SKIP_COPY, 6)
    assert plan.get(st.OPT_TEST_SKIP_COPY) == 6 and plan.get(st.OPT_WAIT_LIMIT) == 2000
    before = st.wait_timeouts()
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, T)
    with pytest.raises(st.StencilError) as e:
        plan.check()
    assert e.value.status == st.ETIMEOUT
    # one CTA gave up in each of the T one-level sweeps
    assert st.wait_timeouts() - before == T
    plan.check()                         # reported once
    # the same plan without the hook: correct again, no timeout
    plan.set(st.OPT_TEST_SKIP_COPY, -1)
    plan.set(st.OPT_WAIT_LIMIT, 0)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    plan.forward(up, u, wk.w, W, T)
    plan.check()
    torch.cuda.synchronize()
    _, ou, _ = oracle.forward(kind, wk.u_prev, wk.u, wk.w, wk.W, T, threads=8)
    assert normwise_err(to_np(u), ou) <= (1e-12 if dtype == F64 else 1e-5)
    plan.close()


@pytest.mark.parametrize("dtype", [F32, F64])
def test_adjoint_wait_gives_up_with_etimeout(st, dtype):
    """The staged adjoint of the 13-array kinds (adjt_kernel) gives up the same way."""
    import torch
    kind, shape, T = wl.W25_VAR, (64, 24, 20), 2
    wk = wl.make(kind, shape, T, seed=6)
    rng = np.random.default_rng(3)
    lam = np.zeros_like(wk.u)
    lam[4:-4, 4:-4, 4:-4] = rng.uniform(-1, 1, size=(shape[2], shape[1], shape[0]))
    plan = st.Plan(kind, *shape, dtype)
    plan.set(st.OPT_VARIANT, 16)
    plan.set(st.OPT_WAIT_LIMIT, 2000)
    plan.set(st.OPT_TEST_SKIP_COPY, 3)
    W = to_dev(wk.W, dtype)
    l2, l1 = to_dev(np.zeros_like(lam), dtype), to_dev(lam, dtype)
    before = st.wait_timeouts()
    plan.adjoint(l2, l1, None, W, T)
    with pytest.raises(st.StencilError) as e:
        plan.check()
    assert e.value.status == st.ETIMEOUT
    assert st.wait_timeouts() - before == T
    plan.set(st.OPT_TEST_SKIP_COPY, -1)
    plan.set(st.OPT_WAIT_LIMIT, 0)
    l2, l1 = to_dev(np.zeros_like(lam), dtype), to_dev(lam, dtype)
    plan.adjoint(l2, l1, None, W, T)
    plan.check()
    torch.cuda.synchronize()
    _, ol1 = oracle.adjoint(kind, np.zeros_like(lam), lam, None, wk.W, T)
    if dtype == F32:
        f32 = lambda a: a.astype(np.float32).astype(np.float64)  # noqa: E731
        _, ol1 = oracle.adjoint(kind, np.zeros_like(lam), f32(lam), None, f32(wk.W), T)
    assert normwise_err(to_np(l1), ol1) <= (1e-12 if dtype == F64 else 1e-5)
    plan.close()
