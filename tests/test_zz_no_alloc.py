"""The allocation-free misfit (stencil_misfit_static) against the plan-based
one (stencil_misfit), through the C ABI, on two calls in a row.

stencil_misfit_static exists for callers that cannot allocate device memory
(an application whose device memory belongs to its own allocator, or a
latency-critical loop that must not allocate): it keeps its partial sums in
a static device array of the library instead of plan scratch.  This file is
collected last so that a run stopping at the first failure has run every
other test first; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def st():
    import torch
    assert torch.cuda.is_available()
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


@pytest.mark.parametrize("dtype", [0, 1])
def test_misfit_static_matches_plan_misfit(st, dtype):
    import torch
    tdt = torch.float64 if dtype == 0 else torch.float32
    T, ny, nx = 9, 37, 51
    plan = st.Plan(4, nx, ny, 16, dtype)
    rng = np.random.default_rng(40 + dtype)
    for call in range(2):   # two calls in a row: nothing may carry over
        tr = torch.from_numpy(rng.uniform(-1, 1, size=(T, ny, nx))).to("cuda", tdt)
        d = torch.from_numpy(rng.uniform(-1, 1, size=(T, ny, nx))).to("cuda", tdt)
        r_ref = torch.empty_like(tr)
        l_ref = torch.zeros(1, device="cuda", dtype=torch.float64)
        plan.misfit(tr, d, r_ref, l_ref)
        r = torch.full_like(tr, float("nan"))
        l = torch.full((1,), float("nan"), device="cuda", dtype=torch.float64)
        st.misfit_static(tr, d, r, l)
        torch.cuda.synchronize()
        assert torch.equal(r, r_ref), call
        rel = abs(l.item() - l_ref.item()) / l_ref.item()
        assert rel <= (1e-13 if dtype == 0 else 1e-6), (call, rel)
    plan.close()


def test_misfit_static_large_and_rejects_beyond_limit(st):
    import torch
    n = 3 * 2048 * 1000 + 17            # many partial sums, ragged tail
    rng = np.random.default_rng(7)
    tr = torch.from_numpy(rng.uniform(-1, 1, size=n)).to("cuda", torch.float64)
    d = torch.zeros_like(tr)
    r = torch.empty_like(tr)
    l = torch.zeros(1, device="cuda", dtype=torch.float64)
    st.misfit_static(tr, d, r, l)
    torch.cuda.synchronize()
    ref = 0.5 * float(np.sum(tr.cpu().numpy() ** 2))
    assert abs(l.item() - ref) <= 1e-12 * ref
    # a size beyond the static scratch is rejected before any launch
    import ctypes
    big = st.MISFIT_STATIC_MAX_ELEMS + 1
    status = st.lib().stencil_misfit_static(0, ctypes.c_void_p(tr.data_ptr()), ctypes.c_void_p(d.data_ptr()), big,
                                            ctypes.c_void_p(r.data_ptr()), ctypes.c_void_p(l.data_ptr()), None)
    assert status == -1
