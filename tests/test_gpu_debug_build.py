"""Sweeps of every kernel family through the debug build (-DSTENCIL_DEBUG,
record-and-skip store checks), the two-level adjoint passes included: no
store leaves the interior of the padded array, and the forward results
still match the oracle.  Runs in a child process
that loads the debug library (STENCIL_LIBRARY)."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import numpy as np, torch, oracle
from paper_1410_3060_gb300 import stencil as st, workloads as wl
from gpu_util import to_dev, to_np, normwise_err, oracle_both, check_fp32
assert st.library_path().endswith("_build_debug/libstencil.so")
cases = []
for kind in (1, 2):
    for b, scheme, variant in ((1, 3, 10), (2, 3, 11), (3, 3, 12), (4, 3, 11), (2, 1, 0), (2, 2, 0), (1, 0, 3)):
        cases.append((kind, st.F32, b, scheme, variant, (70, 45, 23)))
    cases.append((kind, st.F64, 1, 0, 15, (70, 45, 23)))
for kind in (3, 4, 5, 6):
    for variant in (1, 13, 15, 16):
        cases.append((kind, st.F32, 1, 0, variant, (64, 21, 19)))
    cases.append((kind, st.F32, 2, 2, 0, (64, 21, 19)))
for kind in (3, 4, 5):   # the two-level pass (scheme 4)
    cases.append((kind, st.F32, 2, 4, 0, (64, 21, 19)))
T = 5
for kind, dtype, b, scheme, variant, shape in cases:
    wk = wl.make(kind, shape, T, seed=2)
    plan = st.Plan(kind, *shape, dtype)
    plan.set(st.OPT_SCHEME, scheme)
    plan.set(st.OPT_TIME_BLOCK, b)
    plan.set(st.OPT_VARIANT, variant)
    up, u = to_dev(wk.u_prev, dtype), to_dev(wk.u, dtype)
    W = to_dev(wk.W, dtype) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, T)
    plan.check()
    bad = plan.debug_bad_store()
    assert bad == -1, (kind, dtype, b, scheme, variant, bad)
    o64, o32 = oracle_both(wk, T)
    if dtype == st.F64:
        assert normwise_err(to_np(u), o64[1]) <= 1e-12
    else:
        check_fp32((to_np(up), to_np(u)), o64, o32)
    if kind in (2, 4, 5, 6):
        # adjoint with a coefficient gradient
        lam = to_dev(wk.u, dtype)
        lam_next = torch.zeros_like(lam)
        grad = torch.zeros((st.NUM_ARRAYS[kind],) + plan.padded_shape, device="cuda", dtype=torch.float64)
        states = [to_dev(wk.u, dtype) for _ in range(2)]
        plan.adjoint(lam_next, lam, wk.w, W, 2, fwd_states=states, grad=grad)
        plan.check()
        assert plan.debug_bad_store() == -1, ("adjoint", kind, variant)
    if dtype == st.F32 and ((kind in (1, 2) and (b, scheme) == (2, 3)) or (kind in (4, 5) and scheme == 4)):
        # adjoint passes of two levels (gradient batches of 2 steps for the
        # variable kinds): the register wavefront's and the two-level pass's
        plan.set(st.OPT_ADJ_TIME_BLOCK, 2)
        assert plan.get(st.OPT_ADJ_TIME_BLOCK) == 2
        lam = to_dev(wk.u, dtype)
        lam_next = torch.zeros_like(lam)
        grad = states = None
        if st.NUM_ARRAYS[kind]:
            plan.set(st.OPT_GRAD_BATCH, 2)
            grad = torch.zeros((st.NUM_ARRAYS[kind],) + plan.padded_shape, device="cuda", dtype=torch.float64)
            states = [to_dev(wk.u, dtype) for _ in range(4)]
        plan.adjoint(lam_next, lam, wk.w, W, 4, fwd_states=states, grad=grad)
        plan.check()
        assert plan.debug_bad_store() == -1, ("blocked adjoint", kind, scheme)
    plan.close()
print("debug build ok", len(cases))
'''


def test_debug_build_sweeps_store_only_interior_points():
    from paper_1410_3060_gb300 import build
    path = build.build(debug=True)
    env = dict(os.environ, STENCIL_LIBRARY=path, PYTHONPATH=os.pathsep.join([ROOT, os.path.join(ROOT, "tests")]))
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, env=env, cwd=ROOT, timeout=1200)
    assert r.returncode == 0 and "debug build ok" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
