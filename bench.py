"""Benchmark: GLUP/s of the stencil sweeps on one GB300 (and N replicas).

Default workload (one "step"): the 7-point variable-coefficient Jacobi
sweep (paper Fig. 1c), FP64, 512^3 interior + radius-1 zero halo, 7 arrays
~ U[0, 0.14], u0 ~ U[-1, 1], T = 64 time steps through stencil_forward.
value = lattice updates per second (GLUP/s) over all ranks, inputs resident
in HBM; e2e = the same with the state and coefficients copied from pinned
host memory and the final field read back inside the timed region.

Further lines of the same run (key "variants"): the same sweep in FP32
(temporally blocked where the library blocks it), the 25-point constant
and variable wave sweeps (FP64 and FP32), and forward+adjoint.

Timing: CUDA events on the launching stream, a barrier and
torch.cuda.synchronize() on both sides, max over ranks.  Every input is far
larger than the 129 MB L2 (no flush needed).  nvidia-smi clocks are
sampled during the timed region.

--impl reference times the FP64 CPU oracle (the reference arm) on the host
cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "GLUP/s"


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n", type=int, default=512, help="interior size per axis")
    p.add_argument("--T", type=int, default=64, help="time steps per step")
    p.add_argument("--kind", default="j7_var", choices=["j7_const", "j7_var", "w25_const", "w25_var",
                                                          "j25_var", "w25_alpha"])
    p.add_argument("--dtype", default="f64", choices=["f64", "f32"])
    p.add_argument("--time-block", type=int, default=None, help="levels per pass (default: library choice)")
    p.add_argument("--scheme", type=int, default=None,
                   help="1 overlapped tiles, 2 diamond tiles in y, 3 register wavefront")
    p.add_argument("--variant", type=int, default=None, help="plain forward tile variant (0 = default)")
    p.add_argument("--graph", action="store_true", help="replay the captured CUDA graph of the pass program")
    p.add_argument("--sweep", action="store_true", help="time every tile variant and block depth, one line each")
    p.add_argument("--sweep-kinds", default="j7_const,j7_var,w25_const,w25_var",
                   help="comma-separated kinds of the tuning sweep")
    p.add_argument("--sweep-dtypes", default="f64,f32", help="comma-separated dtypes of the tuning sweep")
    p.add_argument("--fwd-adj", action="store_true",
                   help="time only the forward+adjoint of the differentiable workload: the 25-point variable wave "
                        "(K = 20), or --kind j7_var (K = 16) (size --n, T --T)")
    p.add_argument("--adjoint", action="store_true",
                   help="time only the adjoint sweep of a 7-point or 13-array --kind (size --n, T --T, levels "
                        "per pass --time-block, default: library choice)")
    p.add_argument("--no-variants", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    return p.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# --------------------------------------------------------------- reference arm
def cpu_oracle_rate(kind, wk, T_sample, threads, keep=False):
    """GLUP/s and seconds of the FP64 oracle on T_sample steps of the
    workload (and, with keep, its u^T)."""
    import oracle
    t0 = time.perf_counter()
    _, uT, _ = oracle.forward(kind, wk.u_prev, wk.u, wk.w, wk.W, T_sample, threads=threads)
    dt = time.perf_counter() - t0
    n = wk.n[0] * wk.n[1] * wk.n[2]
    return (n * T_sample / dt / 1e9, dt) + ((uT,) if keep else ())


def gpu_one_step_error(torch, st, kind, wk, dtype, oracle_u1):
    """Normwise error (max |g - o| / max |o|) of one GPU step of the plan's
    default program against the oracle's step from the same input."""
    tdt = torch.float64 if dtype == st.F64 else torch.float32
    nx, ny, nz = wk.n
    plan = st.Plan(kind, nx, ny, nz, dtype)
    up = torch.from_numpy(wk.u_prev).to("cuda", tdt)
    u = torch.from_numpy(wk.u).to("cuda", tdt)
    W = torch.from_numpy(wk.W).to("cuda", tdt) if wk.W is not None else None
    plan.forward(up, u, wk.w, W, 1)
    plan.check()
    plan.close()
    o = torch.from_numpy(oracle_u1)
    g = u.to("cpu", torch.float64)
    err = float((g - o).abs().max() / o.abs().max().clamp_min(1e-300))
    del up, u, W
    torch.cuda.empty_cache()
    return err


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (plain C loops of the naive
    sweep, all host cores) on a bounded sample of the same workload -- one
    time step of the full grid per step."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    from paper_1410_3060_gb300 import workloads as wl
    oracle.build()
    threads = oracle.oracle.default_threads()
    kind = KIND_BY_NAME[args.kind]
    wk = wl.make(kind, args.n, args.T, seed=0) if kind != wl.J7_VAR else wl.j7_var(args.n, args.T, seed=0)
    T_sample = 1
    for _ in range(args.warmup):
        cpu_oracle_rate(kind, wk, T_sample, threads)
    rates = [cpu_oracle_rate(kind, wk, T_sample, threads)[0] for _ in range(args.steps)]
    v = statistics.median(rates)
    # the same loops on one core, once (context for the all-core figure)
    v1, dt1 = cpu_oracle_rate(kind, wk, T_sample, 1)
    n3 = args.n ** 3
    sample = f"{T_sample} time step of the {args.n}^3 {args.kind} sweep per step (FP64 plain C loops, {threads} threads)"
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": n3 * T_sample / (v * 1e9) * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.kind}_{args.n}^3_T{args.T}_{args.dtype}", "kind": KIND_TEXT[kind],
                   "n": args.n, "T": args.T, "sample": sample},
        "cpu_baseline": {"value": v, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "cpu_single_thread": {"value": v1, "unit": METRIC, "cores": 1, "kind": "oracle",
                              "sample": f"{T_sample} time step of the {args.n}^3 {args.kind} sweep, once ({dt1:.1f} s)"},
    }
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.dev)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        if not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        # samples under load: top half of the clock samples by power
        ranked = sorted(zip(power, sm), reverse=True)
        top = ranked[:max(1, len(ranked) // 2)]
        load = [s for _, s in top]
        return {"sm_mhz": statistics.median(load), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "power_w_max": max(power),
                "power_w_under_load": statistics.mean(p for p, _ in top)}


# --------------------------------------------------------------- ours
class Timer:
    def __init__(self, torch, stream):
        self.torch, self.stream = torch, stream

    def __enter__(self):
        self.e0 = self.torch.cuda.Event(enable_timing=True)
        self.e1 = self.torch.cuda.Event(enable_timing=True)
        self.e0.record(self.stream)
        return self

    def __exit__(self, *exc):
        self.e1.record(self.stream)
        self.e1.synchronize()
        self.ms = self.e0.elapsed_time(self.e1)


def barrier(torch, ws):
    torch.cuda.synchronize()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()


def max_over_ranks(torch, ws, v):
    """Maximum of a per-rank value over all ranks (the slowest replica sets
    the job time)."""
    if ws == 1:
        return v
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, ws, ms_max):
    """Whole-job throughput: units processed by all ranks / slowest rank's time."""
    return units_per_rank * ws / (ms_max * 1e-3)


def forward_case(torch, st, wl, kind, n, T, dtype, steps, warmup, ws, stream, time_block=None, e2e=False,
                 wk=None, scheme=None, variant=None, graph=False):
    """Time `steps` calls of stencil_forward(T) on the workload; returns dict."""
    tdt = torch.float64 if dtype == st.F64 else torch.float32
    if wk is None:
        wk = wl.make(kind, n, T, seed=0) if kind not in (wl.J7_VAR,) else wl.j7_var(n, T, seed=0)
    plan = st.Plan(kind, n, n, n, dtype)
    if time_block is not None:
        plan.set(st.OPT_TIME_BLOCK, time_block)
    if scheme is not None:
        plan.set(st.OPT_SCHEME, scheme)
    if variant is not None:
        plan.set(st.OPT_VARIANT, variant)
    if graph:
        plan.set(st.OPT_GRAPH, 1)
    b = plan.get(st.OPT_TIME_BLOCK)
    up = torch.from_numpy(wk.u_prev).to("cuda", tdt)
    u = torch.from_numpy(wk.u).to("cuda", tdt)
    W = torch.from_numpy(wk.W).to("cuda", tdt) if wk.W is not None else None
    # every step starts from the workload's initial state (a device copy,
    # restored between steps outside the step's events): the decaying
    # 7-point variable field would otherwise reach zero after a few hundred
    # sweeps, and every step then sweeps the same data
    up0, u0 = up.clone(), u.clone()
    for _ in range(warmup):
        up.copy_(up0)
        u.copy_(u0)
        plan.forward(up, u, wk.w, W, T)
    barrier(torch, ws)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for i in range(steps):
        up.copy_(up0)
        u.copy_(u0)
        ev[i][0].record(stream)
        plan.forward(up, u, wk.w, W, T)
        ev[i][1].record(stream)
    ev[-1][1].synchronize()
    step_ms = sum(a.elapsed_time(b) for a, b in ev)
    barrier(torch, ws)
    ms = max_over_ranks(torch, ws, step_ms)
    del up0, u0
    lups = float(n) ** 3 * T
    passes = [o for o in st.schedule(kind, T, b, dtype) if o[0] == 0]
    res = {"kind": wl.KIND_NAMES[kind], "n": n, "T": T, "dtype": "f64" if dtype == st.F64 else "f32",
           "scheme": plan.get(st.OPT_SCHEME), "variant": plan.get(st.OPT_VARIANT),
           "time_block": b, "ms_per_step": ms / steps, "glups": lups * steps * ws / (ms * 1e-3) / 1e9,
           "launches_per_step": len(passes), "ms_per_launch": ms / steps / len(passes)}
    if e2e:
        hp = torch.from_numpy(wk.u_prev).to(tdt).pin_memory()
        hu = torch.from_numpy(wk.u).to(tdt).pin_memory()
        hW = torch.from_numpy(wk.W).to(tdt).pin_memory() if wk.W is not None else None
        hout = torch.empty_like(hu).pin_memory()
        h2d = hp.numel() * hp.element_size() * 2 + (hW.numel() * hW.element_size() if hW is not None else 0)
        d2h = hout.numel() * hout.element_size()
        # two device input sets: the host->device copy of step i+1's inputs
        # (on one copy stream) and the device->host read of step i-1's result
        # (on another: the link carries both directions at once) run while
        # step i's sweeps run (every step still copies its own inputs and
        # reads its own result inside the timed region)
        sets = [(up, u, W), (torch.empty_like(up), torch.empty_like(u), torch.empty_like(W) if W is not None else None)]
        cs, rs = torch.cuda.Stream(), torch.cuda.Stream()
        copied = [torch.cuda.Event(), torch.cuda.Event()]
        done = [None, None]
        read = [None, None]

        def copy_inputs(k):
            with torch.cuda.stream(cs):
                if done[k] is not None:
                    cs.wait_event(done[k])          # the sweeps that last read this set are finished
                if read[k] is not None:
                    cs.wait_event(read[k])          # and so is the read of their result
                p_, u_, W_ = sets[k]
                p_.copy_(hp, non_blocking=True)
                u_.copy_(hu, non_blocking=True)
                if W_ is not None:
                    W_.copy_(hW, non_blocking=True)
                copied[k].record(cs)

        barrier(torch, ws)
        with Timer(torch, stream) as te:
            cs.wait_stream(stream)
            copy_inputs(0)
            for i in range(steps):
                k = i % 2
                if i + 1 < steps:
                    copy_inputs(1 - k)
                stream.wait_event(copied[k])
                p_, u_, W_ = sets[k]
                plan.forward(p_, u_, wk.w, W_, T, stream=stream)
                ev = torch.cuda.Event()
                ev.record(stream)
                done[k] = ev
                with torch.cuda.stream(rs):
                    rs.wait_event(ev)
                    hout.copy_(u_, non_blocking=True)
                    read[k] = rs.record_event()
            stream.wait_stream(cs)
            stream.wait_stream(rs)
        barrier(torch, ws)
        del sets
        ms_e = max_over_ranks(torch, ws, te.ms)
        res["e2e"] = {"value": lups * steps * ws / (ms_e * 1e-3) / 1e9, "unit": METRIC,
                      "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
    plan.close()
    del up, u, W
    torch.cuda.empty_cache()
    return res, wk


# DRAM bytes per update measured by ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one launch / updates of that launch) for the kernel
# configurations summarised under profiles/, keyed by (kind, dtype, levels per
# pass, tile variant); the roofline record reports them scaled to one launch
# of the benchmarked size, null for any configuration without a profile of
# its current kernel.
MEASURED_TRAFFIC = {
    ("j7_var", "f64", 1, 8): (72.5, "profiles/plain_stream_j7_var_256_fp64.md"),
    ("j7_const", "f32", 3, 12): (2.53, "profiles/wavefront_j7_const_384_fp32_b3_64x64.md"),
    ("j7_var", "f32", 2, 11): (18.47, "profiles/wavefront_j7_var_384_fp32_b2_ring.md"),
    ("w25_var", "f32", 1, 16): (67.88, "profiles/plainv_tma_w25_var_384_fp32.md"),
    ("w25_const", "f32", 1, 15): (12.22, "profiles/plainv_tma_w25_const_512_fp32.md"),
}
# adjoint passes (bench.py --adjoint, no gradient): (kind, dtype, levels)
MEASURED_TRAFFIC_ADJ = {
    ("j7_var", "f32", 2): (18.48, "profiles/wavefront_adj_j7_var_384_fp32_b2.md"),
    ("j7_const", "f32", 2): (3.78, "profiles/wavefront_adj_j7_const_384_fp32_b2.md"),
}


def add_traffic(rec, kind_name, dtype_name, res, n):
    """DRAM traffic per launch of a profiled configuration: the profiled
    bytes per update x the n^3 x levels updates one pass makes."""
    tr = MEASURED_TRAFFIC.get((kind_name, dtype_name, res["time_block"], res["variant"]))
    if tr is not None:
        rec["traffic"] = tr[0] * float(n) ** 3 * res["time_block"]
        rec["traffic_source"] = tr[1] + " (DRAM bytes per update x updates per launch)"
# thread instructions per update of the on-chip-bound FP32 kernels (ncu
# warp instructions x 32 / updates of the profiled launch): the issue view of
# their roofline, ceiling = 4 warp instructions per clock per SM
MEASURED_INSTR = {
    ("j7_const", "f32", 3, 12): (21.9, "profiles/wavefront_j7_const_384_fp32_b3_64x64.md"),
    ("j7_var", "f32", 2, 11): (46.1, "profiles/wavefront_j7_var_384_fp32_b2_ring.md"),
    ("w25_const", "f32", 1, 15): (49.5, "profiles/plainv_tma_w25_const_512_fp32.md"),
}


def issue_view(kind_name, dtype_name, res, num_sms, clk_hz):
    """Instruction-issue ceiling of a profiled kernel configuration, or None."""
    m = MEASURED_INSTR.get((kind_name, dtype_name, res["time_block"], res["variant"]))
    if m is None:
        return None
    ceiling = num_sms * 4 * 32 * clk_hz / m[0] / 1e9
    return {"thread_instr_per_update": m[0], "ceiling_glups": ceiling, "frac": res["glups"] / ceiling,
            "source": m[1]}

KIND_BY_NAME = {"j7_const": 1, "j7_var": 2, "w25_const": 3, "w25_var": 4, "j25_var": 5, "w25_alpha": 6}
KIND_TEXT = {1: "7-point constant coefficients (Fig. 1b)", 2: "7-point variable coefficients (Fig. 1c)",
             3: "25-point constant-coefficient wave (Fig. 1e, scalar alpha)",
             4: "25-point variable-coefficient wave (Fig. 1d coefficients)",
             5: "25-point variable coefficients, first order (Fig. 1d)",
             6: "25-point wave with alpha array (Fig. 1e)"}


def roofline_of(pm, kind, dtype_name, n, res, fp_peaks, hbm_peak):
    """Roofline record of one case (min of ceilings): the HBM ceiling (measured
    copy bandwidth / algorithmic bytes per update) against the FP ceiling
    (the measured FMA-chain rate of the dtype, fp_peaks[dtype]["probe"] in
    flop/s, / flops per update); the lower one is the bound and the record's
    achieved / peak are in its units.  Units processed per pass: n^3 updates
    of `time_block` levels; algorithmic bytes = one read of every input
    stream and one write of the state per pass; flops of every level.  The
    datasheet FP rate (FMA units x SMs x measured clock) is a side view."""
    word = 8 if dtype_name == "f64" else 4
    b = res["time_block"]
    t_pass = res["ms_per_step"] / (res["T"] / b) * 1e-3
    pts = float(n) ** 3
    bytes_pass = pm.gpu_bytes_per_lup(kind, word) * pts
    flops_pass = pm.FLOPS_PER_LUP[kind] * pts * b
    probe, sheet = fp_peaks[dtype_name]["probe"], fp_peaks[dtype_name]["datasheet"]
    hbm_ceiling = hbm_peak * 1e9 / (pm.gpu_bytes_per_lup(kind, word) / b) / 1e9   # GLUP/s
    fp_ceiling = probe / pm.FLOPS_PER_LUP[kind] / 1e9
    hbm = {"achieved_gbs": bytes_pass / t_pass / 1e9, "peak_gbs": hbm_peak,
           "frac": bytes_pass / t_pass / 1e9 / hbm_peak, "ceiling_glups": hbm_ceiling}
    ach_tf = flops_pass / t_pass / 1e12
    fp = {"achieved_tflops": ach_tf, "peak_tflops": probe / 1e12, "frac": ach_tf / (probe / 1e12),
          "ceiling_glups": fp_ceiling, "peak_source": f"measured {dtype_name.upper()} FMA-chain rate",
          "datasheet_peak_tflops": sheet / 1e12, "frac_of_datasheet": ach_tf / (sheet / 1e12),
          # an add occupies a pipe slot like an FMA: the instruction view
          "fp_instr_per_update": pm.FP_INSTR_PER_LUP[kind],
          "instr_frac": pm.FP_INSTR_PER_LUP[kind] * pts * b / t_pass / (probe / 2)}
    if fp_ceiling < hbm_ceiling:
        rec = {"bound": "alu", "achieved": ach_tf, "peak": probe / 1e12, "unit": "TFLOP/s",
               "frac": fp["frac"], "peak_source": fp["peak_source"] + " (stencil_fma_peak)"}
    else:
        rec = {"bound": "hbm", "achieved": hbm["achieved_gbs"], "peak": hbm_peak, "unit": "GB/s",
               "frac": hbm["frac"], "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy, measured)"}
    rec.update({"traffic": None, "ceilings_glups": {"hbm": hbm_ceiling, "fp": fp_ceiling},
                "hbm_view": hbm, "fp_view": fp})
    return rec


def fwd_adj_bytes_per_lup(elem, T, K, grad_batch):
    """Algorithmic HBM bytes per lattice update of one forward + backward of
    the 25-point variable wave: the forward sweep, the recompute of every
    segment but the last (whose states the forward pass keeps) and the
    adjoint sweep each read two fields and the 13 coefficient arrays and
    write one field; the gradient reads the adjoint level and the state of
    every step and reads and writes the 13 FP64 gradient arrays once per
    batch of grad_batch steps."""
    sweep = 16 * elem
    nseg = (T + K - 1) // K
    recomputed = (T - (T - (nseg - 1) * K)) / T
    return sweep * (2 + recomputed) + 2 * elem + 13 * 16 / grad_batch


def fwd_adj_j7_bytes_per_lup(elem, T, K, grad_batch, levels):
    """Algorithmic HBM bytes per lattice update of one forward + backward of
    the 7-point variable kind with passes of `levels` levels (forward,
    recompute and adjoint): the forward reads the state and the 7 arrays and
    writes the last level once per pass; the recompute of every segment but
    the last and the adjoint write every level; the gradient reads the
    adjoint level and the state of every step and reads and writes the 7
    FP64 gradient arrays once per batch."""
    b = levels
    fwd = elem * (1 + 7 + 1) / b
    every = elem * (1 + 7 + b) / b
    nseg = (T + K - 1) // K
    recomputed = (T - (T - (nseg - 1) * K)) / T
    return fwd + every * recomputed + every + 2 * elem + 7 * 16 / grad_batch


def fwd_adj_j7_case(torch, st, wl, n, T, K, dtype, steps, warmup, ws, stream, hbm_peak=None):
    """Differentiable 7-point variable workload through MisfitRunner: one step
    = the checkpointed forward (T steps, state kept every K steps, receiver
    trace on plane n/8, FP64 misfit) plus the backward (recompute and
    adjoint with the FP64 coefficient gradient in 16-step batches).  Inputs:
    the standard 7-point variable recipe (U[-1,1] field, U[0,0.14] weights);
    the observed data come from a forward run of the same library with the
    weights scaled by 1 + 0.05 U[-1,1] (on the device)."""
    from paper_1410_3060_gb300.autograd import MisfitRunner
    tdt = torch.float64 if dtype == st.F64 else torch.float32
    wk = wl.j7_var(n, 1, seed=0)
    rz = max(1, n // 8)
    run = MisfitRunner(wl.J7_VAR, (n, n, n), T, K, rz, dtype=dtype)
    u0 = torch.from_numpy(wk.u).to("cuda", tdt)
    W = torch.from_numpy(wk.W).to("cuda", tdt)
    del wk
    g = torch.Generator(device="cuda")
    g.manual_seed(3)
    Wt = W * (1.0 + 0.05 * (2.0 * torch.rand(W.shape, device="cuda", generator=g, dtype=tdt) - 1.0))
    d = torch.zeros((T, n, n), device="cuda", dtype=tdt)
    up, uc = u0.clone(), u0.clone()
    run.plan.forward(up, uc, None, Wt, T, trace=d, rcv_z=rz)
    del up, uc, Wt

    for _ in range(warmup):
        loss, state = run.forward_pass(u0, W, d)
        run.backward_pass(state, W, torch.ones((), dtype=torch.float64))
        del state
    barrier(torch, ws)
    t_f = t_b = 0.0
    for _ in range(steps):
        with Timer(torch, stream) as tf:
            loss, state = run.forward_pass(u0, W, d)
        with Timer(torch, stream) as tb:
            run.backward_pass(state, W, torch.ones((), dtype=torch.float64))
        t_f += tf.ms
        t_b += tb.ms
        del state
    barrier(torch, ws)
    ms = max_over_ranks(torch, ws, (t_f + t_b) / steps)
    lups = float(n) ** 3 * T
    b = run.plan.get(st.OPT_TIME_BLOCK)
    ab = run.plan.get(st.OPT_ADJ_TIME_BLOCK)
    res = {"kind": "j7_var_fwd_adj", "n": n, "T": T, "K": K, "dtype": "f64" if dtype == st.F64 else "f32",
           "ms_per_step": ms, "glups": lups * ws / (ms * 1e-3) / 1e9,
           "forward_ms": t_f / steps, "backward_ms": t_b / steps,
           "forward_glups": lups / (t_f / steps * 1e-3) / 1e9, "loss": float(loss.item()),
           "time_block": b, "adjoint_levels_per_pass": ab, "grad_batch": run.plan.get(st.OPT_GRAD_BATCH)}
    if hbm_peak and b == ab:
        bpl = fwd_adj_j7_bytes_per_lup(4 if dtype == st.F32 else 8, T, K, res["grad_batch"], b)
        ach = res["glups"] / ws * bpl
        res["roofline"] = {"bound": "hbm", "bytes_per_lup": bpl, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                           "frac": ach / hbm_peak,
                           "note": "algorithmic bytes of forward + recompute + adjoint + gradient"}
    run.close()
    del u0, W, d
    torch.cuda.empty_cache()
    return res


def fwd_adj_case(torch, st, wl, n, T, K, dtype, steps, warmup, ws, stream, fw=None, variant=None, hbm_peak=None):
    """Differentiable 25-point variable wave workload: one step = the
    checkpointed forward (T steps, state pair kept every K steps, receiver
    trace, FP64 misfit) plus the backward (recompute of every segment and the
    adjoint sweep with FP64 coefficient gradients) through MisfitRunner.
    GLUP/s = n^3 T / (forward + backward time).  The observed data come from a
    forward run of the same library with the perturbed model."""
    from paper_1410_3060_gb300.autograd import MisfitRunner
    tdt = torch.float64 if dtype == st.F64 else torch.float32
    if fw is None:
        fw = wl.fwi(n, T=T, K=K, seed=0)
    nx, ny, nz = fw.n
    run = MisfitRunner(wl.W25_VAR, fw.n, T, K, fw.rcv_z, dtype=dtype)
    if variant is not None:
        run.plan.set(st.OPT_VARIANT, variant)
    u0 = torch.from_numpy(fw.u0).to("cuda", tdt)
    W = torch.from_numpy(fw.W).to("cuda", tdt)
    Wt = torch.from_numpy(fw.W_true).to("cuda", tdt)
    d = torch.zeros((T, ny, nx), device="cuda", dtype=tdt)
    up, uc = u0.clone(), u0.clone()
    run.plan.forward(up, uc, None, Wt, T, trace=d, rcv_z=fw.rcv_z)
    del up, uc, Wt

    def one():
        loss, state = run.forward_pass(u0, W, d)
        du0, dW = run.backward_pass(state, W, torch.ones((), dtype=torch.float64))
        return loss, du0, dW

    for _ in range(warmup):
        one()
    barrier(torch, ws)
    t_f = t_b = 0.0
    for _ in range(steps):
        with Timer(torch, stream) as tf:
            loss, state = run.forward_pass(u0, W, d)
        with Timer(torch, stream) as tb:
            run.backward_pass(state, W, torch.ones((), dtype=torch.float64))
        t_f += tf.ms
        t_b += tb.ms
        del state
    barrier(torch, ws)
    ms = max_over_ranks(torch, ws, (t_f + t_b) / steps)
    lups = float(nx) * ny * nz * T
    res = {"kind": "w25_var_fwd_adj", "n": n, "T": T, "K": K, "dtype": "f64" if dtype == st.F64 else "f32",
           "ms_per_step": ms, "glups": lups * ws / (ms * 1e-3) / 1e9,
           "forward_ms": t_f / steps, "backward_ms": t_b / steps,
           "forward_glups": lups / (t_f / steps * 1e-3) / 1e9, "loss": float(loss.item()),
           "time_block": run.plan.get(st.OPT_TIME_BLOCK), "variant": run.plan.get(st.OPT_VARIANT)}
    if hbm_peak:
        bpl = fwd_adj_bytes_per_lup(4 if dtype == st.F32 else 8, T, K, run.plan.get(st.OPT_GRAD_BATCH))
        ach = res["glups"] / ws * bpl
        res["roofline"] = {"bound": "hbm", "bytes_per_lup": bpl, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                           "frac": ach / hbm_peak,
                           "note": "algorithmic bytes of forward + recompute + adjoint + gradient"
                                   + ("" if dtype == st.F32 else "; FP64 is bound by the FP64 pipe")}
    run.close()
    del u0, W, d
    torch.cuda.empty_cache()
    return res, fw


def adjoint_bytes_per_lup(kind, elem, levels):
    """Algorithmic HBM bytes per update of the adjoint sweep of a 7-point
    kind without a gradient: a pass of `levels` levels reads lam^{t+1} and
    the coefficient arrays once and writes its last level (with a gradient
    every level is written, one more field per extra level)."""
    arrays = 7 if kind == 2 else 0
    return elem * (2 + arrays) / levels


def adjoint_case(torch, st, wl, kind, n, T, dtype, steps, warmup, ws, stream, adj_block=None, hbm_peak=None):
    """The adjoint sweep of a 7-point or 13-array kind: one step = T adjoint levels of the
    n^3 lattice with a residual plane injected at every level (no
    gradient), lam reset from a device copy before every step (outside the
    events).  GLUP/s = n^3 T / time."""
    tdt = torch.float64 if dtype == st.F64 else torch.float32
    wk = wl.make(kind, n, 1, seed=0) if kind != wl.J7_VAR else wl.j7_var(n, 1, seed=0)
    plan = st.Plan(kind, n, n, n, dtype)
    if adj_block is not None:
        plan.set(st.OPT_ADJ_TIME_BLOCK, adj_block)
    r7 = kind in (wl.J7_CONST, wl.J7_VAR)
    W = torch.from_numpy(wk.W).to("cuda", tdt) if wk.W is not None else None
    lam0 = torch.from_numpy(wk.u).to("cuda", tdt)
    l2, l1 = torch.zeros_like(lam0), lam0.clone()
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    res = torch.rand((T, n, n), device="cuda", generator=g, dtype=tdt)
    rz = n // 3

    def one():
        plan.adjoint(l2, l1, wk.w, W, T, residual=res, rcv_z=rz, stream=stream)

    for _ in range(warmup):
        l2.zero_()
        l1.copy_(lam0)
        one()
    barrier(torch, ws)
    tot = 0.0
    for _ in range(steps):
        l2.zero_()
        l1.copy_(lam0)
        with Timer(torch, stream) as t:
            one()
        tot += t.ms
    barrier(torch, ws)
    plan.check()
    ms = max_over_ranks(torch, ws, tot / steps)
    lups = float(n) ** 3 * T
    b = plan.get(st.OPT_ADJ_TIME_BLOCK)
    res_ = {"kind": wl.KIND_NAMES[kind] + "_adjoint", "n": n, "T": T, "dtype": "f64" if dtype == st.F64 else "f32",
            "adjoint_levels_per_pass": b, "ms_per_step": ms, "glups": lups * ws / (ms * 1e-3) / 1e9,
            "variant": plan.get(st.OPT_VARIANT)}
    if hbm_peak and r7:   # the 13-array kinds' passes are latency-bound: no byte roofline stated
        bpl = adjoint_bytes_per_lup(kind, 4 if dtype == st.F32 else 8, b)
        ach = res_["glups"] / ws * bpl
        res_["roofline"] = {"bound": "hbm", "bytes_per_lup": bpl, "achieved": ach, "peak": hbm_peak, "unit": "GB/s",
                            "frac": ach / hbm_peak,
                            "note": "algorithmic bytes: lam^{t+1} and the coefficients read, the last level written, once per pass"}
        tr = MEASURED_TRAFFIC_ADJ.get((wl.KIND_NAMES[kind], res_["dtype"], b))
        if tr is not None:
            res_["roofline"]["traffic"] = tr[0] * float(n) ** 3 * b
            res_["roofline"]["traffic_source"] = tr[1] + " (DRAM bytes per update x updates per launch)"
    plan.close()
    del W, lam0, l1, l2, res
    torch.cuda.empty_cache()
    return res_


def run_sweep(args, torch, st, wl, pm, stream, ws, fp_peaks, hbm_peak):
    """Tuning sweep (the auto-tuning of tile parameters): every forward tile
    variant and block depth of every kind and dtype at the given size; one
    JSON line per case."""
    n, T = args.n, args.T
    from paper_1410_3060_gb300 import tune
    kinds = [KIND_BY_NAME[k] for k in args.sweep_kinds.split(",") if k]
    dtypes = [st.F64 if d == "f64" else st.F32 for d in args.sweep_dtypes.split(",") if d]

    def model_of(kind, dtype, b, scheme, variant):
        # the GPU block model's record of the configuration (tune.model_candidates)
        for cb, cs, cv, m in tune.model_candidates(kind, dtype):
            if (cb, cs, cv) == (b, scheme or 0, variant or 0) or (b == 1 and cb == 1 and cv == variant):
                return {k: (list(v) if isinstance(v, tuple) else v) for k, v in m.items()}
        return None

    for kind in kinds:
        wk = wl.make(kind, n, T, seed=0) if kind != wl.J7_VAR else wl.j7_var(n, T, seed=0)
        r1 = wl.RADIUS[kind] == 1
        for dtype in dtypes:
            wide = (17,) if r1 and dtype == st.F32 else ()
            for v in (1, 2, 3, 4, 5, 6, 7, 8, 9) + ((10, 11, 12, 13, 14, 15, 16) if r1 else (13, 14, 15, 16)) + wide:
                r, _ = forward_case(torch, st, wl, kind, n, T, dtype, args.steps, 1, ws, stream, time_block=1,
                                    wk=wk, variant=v)
                r["roofline"] = roofline_of(pm, kind, r["dtype"], n, r, fp_peaks, hbm_peak)
                r["model"] = model_of(kind, dtype, 1, 0, r["variant"])
                print(json.dumps({"sweep": r}), flush=True)
            blocked = ((2, 3, 4) if r1 else (2,)) if dtype == st.F32 else ((2,) if r1 else ())
            for b in blocked:
                cases = [(1, None), (2, None)] + ([(3, 10), (3, 11), (3, 12)] if r1 else []) + \
                    ([(3, 17)] if r1 and dtype == st.F32 else [])
                for sch, v in cases:
                    r, _ = forward_case(torch, st, wl, kind, n, T, dtype, args.steps, 1, ws, stream,
                                        time_block=b, wk=wk, scheme=sch, variant=v)
                    r["roofline"] = roofline_of(pm, kind, r["dtype"], n, r, fp_peaks, hbm_peak)
                    r["model"] = model_of(kind, dtype, r["time_block"], sch, v)
                    print(json.dumps({"sweep": r}), flush=True)
        del wk


def run_ours(args):
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    from paper_1410_3060_gb300 import perfmodel as pm, stencil as st, workloads as wl
    st.lib()
    stream = torch.cuda.current_stream()
    n, T = args.n, args.T
    kind = KIND_BY_NAME[args.kind]
    dtype = st.F64 if args.dtype == "f64" else st.F32

    probe_f64, clk = st.fma_peak(st.F64)
    probe_f32, _ = st.fma_peak(st.F32)
    num_sms = torch.cuda.get_device_properties(0).multi_processor_count
    sheet_f64 = 2 * 2 * num_sms * clk      # datasheet: 2 FP64 FMA per clock per SM (GB300)
    sheet_f32 = 2 * 128 * num_sms * clk    # datasheet: 128 FP32 FMA per clock per SM
    fp_peaks = {"f64": {"probe": probe_f64, "datasheet": sheet_f64},
                "f32": {"probe": probe_f32, "datasheet": sheet_f32}}
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
        os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    hbm_peak = peaks.get("hbm_gbs", 6800.0)

    if args.sweep:
        run_sweep(args, torch, st, wl, pm, stream, ws, fp_peaks, hbm_peak)
        return
    if args.fwd_adj and kind == wl.J7_VAR:
        r = fwd_adj_j7_case(torch, st, wl, n, T, 16, dtype, args.steps, args.warmup, ws, stream, hbm_peak=hbm_peak)
        print(json.dumps({"fwd_adj": r}), flush=True)
        return
    if args.fwd_adj:
        r, _ = fwd_adj_case(torch, st, wl, n, T, 20, dtype, args.steps, args.warmup, ws, stream,
                            variant=args.variant, hbm_peak=hbm_peak)
        print(json.dumps({"fwd_adj": r}), flush=True)
        return
    if args.adjoint:
        if kind not in (wl.J7_CONST, wl.J7_VAR, wl.W25_VAR, wl.J25_VAR):
            raise SystemExit("--adjoint: a 7-point kind or a 13-array kind (j7_const, j7_var, w25_var, j25_var)")
        r = adjoint_case(torch, st, wl, kind, n, T, dtype, args.steps, args.warmup, ws, stream,
                         adj_block=args.time_block, hbm_peak=hbm_peak)
        print(json.dumps({"adjoint": r}), flush=True)
        return
    dev_index = torch.cuda.current_device()
    sampler = ClockSampler(dev_index)
    wk = wl.make(kind, n, T, seed=0) if kind != wl.J7_VAR else wl.j7_var(n, T, seed=0)
    with sampler:
        main, _ = forward_case(torch, st, wl, kind, n, T, dtype, args.steps, args.warmup, ws, stream,
                               time_block=args.time_block, e2e=not args.no_e2e, wk=wk, scheme=args.scheme,
                               variant=args.variant, graph=args.graph)
    clocks = sampler.summary()
    roofline = roofline_of(pm, kind, args.dtype, n, main, fp_peaks, hbm_peak)
    add_traffic(roofline, args.kind, args.dtype, main, n)
    if main["time_block"] == 1 and 13 <= main["variant"] <= 16:
        kname = "plainv_kernel (vectorised, " + ("TMA" if main["variant"] >= 15 else "cp.async") + " staging)"
    elif main["scheme"] == 3 or 10 <= main["variant"] <= 12:
        kname = f"wavefront_kernel (register wavefront, {main['time_block']} levels per pass)"
    elif main["time_block"] == 1:
        kname = "plain_stream_kernel" if main["variant"] != 5 else "plain_sweep_kernel"
    else:
        kname = "blocked_kernel (phase A + B)" if main["scheme"] == 2 else "blocked_kernel (overlapped)"
    roofline["kernel"] = kname + f"<{'double' if dtype == st.F64 else 'float'}, {args.kind}>"
    iv = issue_view(args.kind, args.dtype, main, num_sms, clk)
    if iv:
        roofline["issue_view"] = iv

    variants = []
    if not args.no_variants:
        cases = [(wl.J7_VAR, st.F32, T, 1), (wl.J7_VAR, st.F32, T, None),
                 (wl.W25_CONST, st.F64, 100, 1), (wl.W25_CONST, st.F32, 100, 1), (wl.W25_CONST, st.F32, 100, None),
                 (wl.W25_VAR, st.F64, T, 1), (wl.W25_VAR, st.F32, T, 1), (wl.W25_VAR, st.F32, T, None),
                 (wl.J7_CONST, st.F64, T, 1), (wl.J7_CONST, st.F32, T, 1), (wl.J7_CONST, st.F32, T, None)]
        cache = {wl.J7_VAR: wk} if kind == wl.J7_VAR else {}
        for vk, vd, vT, vb in cases:
            if vk not in cache:
                cache.clear()
                cache[vk] = wl.make(vk, n, vT, seed=0) if vk != wl.J7_VAR else wl.j7_var(n, vT, seed=0)
            r, _ = forward_case(torch, st, wl, vk, n, vT, vd, max(1, args.steps // 2), 1, ws, stream,
                                time_block=vb, wk=cache[vk])
            r["roofline"] = roofline_of(pm, vk, r["dtype"], n, r, fp_peaks, hbm_peak)
            add_traffic(r["roofline"], wl.KIND_NAMES[vk], r["dtype"], r, n)
            iv = issue_view(wl.KIND_NAMES[vk], r["dtype"], r, num_sms, clk)
            if iv:
                r["roofline"]["issue_view"] = iv
            variants.append(r)
        cache.clear()
        # adjoint sweeps of the 7-point kinds (FP32): two levels per pass (the
        # default) and one
        for vk in (wl.J7_VAR, wl.J7_CONST):
            for ab in (None, 1):
                variants.append(adjoint_case(torch, st, wl, vk, n, T, st.F32, max(1, args.steps // 2), 1, ws,
                                             stream, adj_block=ab, hbm_peak=hbm_peak))
        # forward + adjoint of the differentiable 7-point variable workload
        # (512^3, T = 64, K = 16, FP32: blocked forward, recompute and adjoint)
        variants.append(fwd_adj_j7_case(torch, st, wl, n, T, 16, st.F32, 1, 1, ws, stream, hbm_peak=hbm_peak))
        # forward + adjoint of the differentiable wave workload (256^3, T = 200, K = 20)
        fw = None
        for vd in (st.F32, st.F64):
            r, fw = fwd_adj_case(torch, st, wl, 256, 200, 20, vd, 1, 1, ws, stream, fw=fw, hbm_peak=hbm_peak)
            variants.append(r)

    cpu = None
    max_rel_err = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        threads = oracle.oracle.default_threads()
        rate, dt, o1 = cpu_oracle_rate(kind, wk, 1, threads, keep=True)
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle",
               "sample": f"1 time step of the {n}^3 {args.kind} FP64 sweep ({dt:.1f} s)"}
        # the GPU's first step against this oracle step (the full-T errors
        # are measured by tests/test_gpu_errors.py)
        max_rel_err = {"value": gpu_one_step_error(torch, st, kind, wk, dtype, o1), "T": 1,
                       "metric": "max |gpu - oracle| / max |oracle| of u^1, whole 512^3 lattice",
                       "vs": "FP64 oracle step of the cpu_baseline sample"}
        del o1

    if rank == 0:
        line = {
            "metric": METRIC, "value": main["glups"], "unit": METRIC, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": args.dtype, "data": "synthetic",
            "config": {"workload": f"{args.kind}_{n}^3_T{T}_{args.dtype}", "kind": KIND_TEXT[kind],
                       "n": n, "T": T, "time_block": main["time_block"], "parallelism": f"replicas{ws}",
                       "l2": "inputs larger than L2 (no flush needed)" if n >= 256 else "small case",
                       "state": "reset to u0 from a device copy before every step, outside the step's events"},
            "e2e": main.get("e2e"), "gpu_launches": main["launches_per_step"] * args.steps,
            "roofline": roofline, "clocks": clocks, "cpu_baseline": cpu, "max_rel_err": max_rel_err,
            "energy": ({"joules_per_step": clocks["power_w_under_load"] * main["ms_per_step"] * 1e-3,
                        "nJ_per_lup": clocks["power_w_under_load"] * main["ms_per_step"] * 1e-3
                        / (float(n) ** 3 * T) * 1e9,
                        "method": "mean nvidia-smi board power of the loaded half of the samples x time per step"}
                       if clocks.get("power_w_under_load") else None),
            "peaks_measured": {"fp64_fma_probe_tflops": probe_f64 / 1e12, "fp32_fma_probe_tflops": probe_f32 / 1e12,
                               "fp64_datasheet_tflops": sheet_f64 / 1e12, "fp32_datasheet_tflops": sheet_f32 / 1e12,
                               "sm_clock_mhz": clk / 1e6, "hbm_gbs": hbm_peak},
            "variants": variants,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
