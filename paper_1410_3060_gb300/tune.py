"""Run-time tuning of a plan's pass kernels: the GPU analogue of the paper's
auto-tuning of the wavefront-diamond tile parameters (Sect. 5.1), whose
search space is narrowed to the tiles whose cache block fits the cache
(Sect. 5.3).

Candidates are (time block b, scheme, tile variant) triples.  The GPU block
model (perfmodel.wavefront_block, perfmodel.vector_sweep_block: a CTA's
shared memory and register ring against 227 KB and the register file, and
the redundancy of its overlapped halo) proposes them, drops those that do
not fit, and orders the rest by modelled HBM bytes per update (fewest
first; then the least redundant tile).  Families the model does not describe
(the streaming tiles 1-9 and the shared-memory blocked schemes 1 and 2)
follow, in the model's byte order as well.  Each candidate is then timed on
the caller's own data with CUDA events -- the measurement decides, as in the
paper.  A candidate the library rejects is skipped.  The trial runs advance
copies of the caller's state, never the caller's buffers.  tune_adjoint
does the same for the levels per adjoint pass (1 or 2).
"""
from __future__ import annotations

from . import perfmodel as pm
from . import stencil as st


def model_candidates(kind: int, dtype: int):
    """[(b, scheme, variant, model)] for the kind and dtype: the register
    wavefront (7-point kinds) at every depth and tile, the vectorised sweep
    tiles (one level), the streaming tiles and the shared-memory blocked
    schemes, each with its model record; infeasible ones removed, the rest
    ordered by modelled HBM bytes per update, then redundancy."""
    word = 8 if dtype == st.F64 else 4
    r1 = st.RADIUS[kind] == 1
    out = []
    depths = (1, 2, 3, 4) if dtype == st.F32 else (1, 2)
    if r1:
        for b in depths:
            for v in pm.WF_VARIANTS:
                if v in pm.WF_VARIANTS_WIDE and word != 4:
                    continue
                m = pm.wavefront_block(kind, word, b, v)
                m["family"] = "register wavefront"
                out.append((b, 3, v, m))
    for v in (13, 14, 15, 16):
        if r1 and word == 4:
            continue          # FP32 7-point rows are not 16-byte aligned
        m = pm.vector_sweep_block(kind, word, v)
        m["family"] = "vectorised sweep" + (" (TMA)" if v >= 15 else "")
        out.append((1, 0, v, m))
    for v in range(1, 10):
        out.append((1, 0, v, {"family": "streaming tile", "fits": True, "redundancy": 1.0}))
    if kind in (st.W25_VAR, st.J25_VAR, st.W25_CONST) and dtype == st.F32:
        m = pm.two_level_block(kind)
        m["family"] = "two-level 13-array pass"
        out.append((2, 4, 0, m))
    blocked = ((2, 3, 4) if r1 else (2,)) if dtype == st.F32 else ((2,) if r1 else ())
    for b in blocked:
        for s in (1, 2):
            out.append((b, s, 0, {"family": "shared-memory blocked", "fits": True, "redundancy": None}))
    for b, s, v, m in out:
        m["dram_bytes_per_lup"] = pm.dram_bytes_per_lup(kind, word, b)
    keep = [c for c in out if c[3]["fits"]]
    keep.sort(key=lambda c: (c[3]["dram_bytes_per_lup"], c[3]["redundancy"] or 1e9))
    return keep


def default_candidates(plan: st.Plan):
    """(b, scheme, variant) triples of model_candidates for the plan (every
    one-level tile variant and every blocked configuration when no plan is
    given)."""
    if plan is None:
        out = [(1, 0, v) for v in range(1, 18)]
        for b in (2, 3, 4):
            out += [(b, 3, v) for v in pm.WF_VARIANTS]
            out += [(b, s, 0) for s in (1, 2)]
        return out
    return [(b, s, v) for b, s, v, _ in model_candidates(plan.kind, plan.dtype)]


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


def tune_adjoint(plan: st.Plan, lam_next, lam, w=None, W=None, T: int = 8, fwd_states=None, residual=None,
                 rcv_z: int = 0, grad=None, reps: int = 2, stream=None):
    """Time stencil_adjoint(T) with one and with two levels per pass (where
    the plan serves two) on copies of (lam_next, lam) and, when a gradient
    is asked for, into a scratch gradient (the caller's buffers are never
    written); set the faster depth on the plan (STENCIL_OPT_ADJ_TIME_BLOCK)
    and return {"adjoint_levels_per_pass", "ms", "table": [(ms, levels), ...]}.
    The plan must be idle (options are changed between trials)."""
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    tn, tl = lam_next.clone(), lam.clone()
    tg = torch.zeros_like(grad) if grad is not None else None
    table = []
    for b in (1, 2):
        try:
            plan.set(st.OPT_ADJ_TIME_BLOCK, b)
        except st.StencilError:
            continue                      # depth not served for this kind / dtype / geometry
        if plan.get(st.OPT_ADJ_TIME_BLOCK) != b:
            continue

        def run():
            tn.copy_(lam_next)
            tl.copy_(lam)
            plan.adjoint(tn, tl, w, W, T, fwd_states=fwd_states, residual=residual, rcv_z=rcv_z, grad=tg,
                         stream=s)

        run()                             # warm-up (and first-use setup)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            run()
        e1.record(s)
        e1.synchronize()
        table.append((e0.elapsed_time(e1) / reps, b))
    if not table:
        raise RuntimeError("no adjoint depth ran")
    ms, b = min(table)
    plan.set(st.OPT_ADJ_TIME_BLOCK, b)
    del tn, tl, tg
    return {"adjoint_levels_per_pass": b, "ms": ms, "table": sorted(table)}
