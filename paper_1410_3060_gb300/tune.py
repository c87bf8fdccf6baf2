"""Run-time tuning of a plan's pass kernels: the analogue of the paper's
auto-tuning of the wavefront-diamond tile parameters (Sect. 5.1, the block
size model of Sect. 5.3 giving the candidates), done by timing each candidate
on the caller's own data with CUDA events.

Candidates are (time block b, scheme, tile variant) triples the library
accepts for the plan; a candidate the library rejects is skipped.  The trial
runs advance copies of the caller's state, never the caller's buffers.
"""
from __future__ import annotations

from . import stencil as st


def default_candidates(plan: st.Plan):
    """Every one-level tile variant, and every block depth with every blocked
    kernel family (register wavefront tiles, shared-memory overlapped and
    diamond tiles)."""
    out = [(1, 0, v) for v in range(1, 17)]
    for b in (2, 3, 4):
        out += [(b, 3, v) for v in (10, 11, 12)]
        out += [(b, s, 0) for s in (1, 2)]
    return out


def tune_forward(plan: st.Plan, u_prev, u, w=None, W=None, T: int = 8, candidates=None, reps: int = 2,
                 stream=None):
    """Time stencil_forward(T) for each candidate on copies of (u_prev, u);
    set the fastest on the plan and return
    {"time_block", "scheme", "variant", "ms", "table": [(ms, b, scheme, variant), ...]}.
    The plan must be idle (options are changed between trials)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    tp, tu = u_prev.clone(), u.clone()
    table = []
    for b, scheme, variant in (candidates or default_candidates(plan)):
        try:
            plan.set(st.OPT_TIME_BLOCK, b)
            plan.set(st.OPT_SCHEME, scheme)
            plan.set(st.OPT_VARIANT, variant)
        except st.StencilError:
            continue
        if plan.get(st.OPT_TIME_BLOCK) != b:
            continue                      # depth not served for this scheme / geometry
        tp.copy_(u_prev)
        tu.copy_(u)
        plan.forward(tp, tu, w, W, T, stream=s)          # warm-up (and first-use setup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            plan.forward(tp, tu, w, W, T, stream=s)
        e1.record(s)
        e1.synchronize()
        table.append((e0.elapsed_time(e1) / reps, b, scheme, variant))
    if not table:
        raise RuntimeError("no candidate configuration ran")
    ms, b, scheme, variant = min(table)
    plan.set(st.OPT_TIME_BLOCK, b)
    plan.set(st.OPT_SCHEME, scheme)
    plan.set(st.OPT_VARIANT, variant)
    del tp, tu
    return {"time_block": b, "scheme": scheme, "variant": variant, "ms": ms, "table": sorted(table)}
