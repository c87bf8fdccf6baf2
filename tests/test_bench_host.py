"""Host logic of bench.py and the run-time tuner (no GPU): the roofline
record's arithmetic and the tuner's candidate list."""
import importlib.util
import os

import pytest

from paper_1410_3060_gb300 import perfmodel as pm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_fp32_roofline_counts_bytes_once_per_pass(bench):
    """A pass of b levels moves the plain bytes of one update once: at 64
    steps in 16 passes of 4 levels taking 1 s in total, 512^3 points x 36 B
    x 16 passes of 7-point variable FP32 traffic per second."""
    n, T, b, ms = 512, 64, 4, 1000.0
    res = {"time_block": b, "ms_per_step": ms, "T": T}
    peaks = {"f32": {"probe": 70e12, "datasheet": 80e12}, "f64": {"probe": 1.05e12, "datasheet": 1.26e12}}
    r = bench.roofline_of(pm, pm.J7_VAR, "f32", n, res, peaks, 6788.6)
    expect_gbs = 36.0 * n ** 3 * (T / b) / 1.0 / 1e9
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert abs(r["achieved"] - expect_gbs) < 1e-9 * expect_gbs
    assert abs(r["frac"] - expect_gbs / 6788.6) < 1e-12
    # ceilings: HBM 6788.6 GB/s / (36 B / 4 levels); FP 70 TFLOP/s / 13 flops
    assert abs(r["ceilings_glups"]["hbm"] - 6788.6 / 9.0) < 1e-9
    assert abs(r["ceilings_glups"]["fp"] - 70e3 / 13) < 1e-6


def test_fwd_adj_bytes_per_update(bench):
    """Forward + backward of the 25-point variable wave, FP32, T = 200 in
    segments of 20 (the last kept, 180 steps recomputed), gradient batches of
    16: 64 B forward + 0.9 x 64 B recompute + 64 B adjoint + 8 B gradient
    reads + 13 x 16 / 16 B of FP64 read-modify-write per update."""
    assert abs(bench.fwd_adj_bytes_per_lup(4, 200, 20, 16) - (64 + 57.6 + 64 + 8 + 13)) < 1e-12
    # one segment: nothing is recomputed
    assert abs(bench.fwd_adj_bytes_per_lup(8, 20, 20, 1) - (128 + 128 + 16 + 208)) < 1e-12


def test_fp64_roofline_takes_the_lower_ceiling(bench):
    """FP64: the bound is the lower of the HBM ceiling and the FP ceiling of
    the measured FMA-chain rate.  7-point variable (72 B, 13 flops per
    update): HBM 6788.6 / 72 = 94.3 GLUP/s, FP 1.054e12 / 13 = 81.1 -> FP
    bound; the datasheet rate and the instruction view are side views."""
    n, T, ms = 512, 64, 1000.0
    probe, sheet = 1.054e12, 1.2544e12
    peaks = {"f64": {"probe": probe, "datasheet": sheet}, "f32": {"probe": 70e12, "datasheet": 80e12}}
    res = {"time_block": 1, "ms_per_step": ms, "T": T}
    r = bench.roofline_of(pm, pm.J7_VAR, "f64", n, res, peaks, 6788.6)
    lups = float(n) ** 3 * T
    assert r["bound"] == "alu" and r["unit"] == "TFLOP/s"
    assert abs(r["achieved"] - 13 * lups / 1e12) < 1e-9
    assert abs(r["peak"] - probe / 1e12) < 1e-12 and abs(r["frac"] - 13 * lups / probe) < 1e-12
    fv = r["fp_view"]
    assert fv["fp_instr_per_update"] == 7
    assert abs(fv["instr_frac"] - 7 * lups / (probe / 2)) < 1e-12
    assert abs(fv["frac_of_datasheet"] - 13 * lups / sheet) < 1e-12
    # a fast FP64 pipe would leave HBM as the bound
    peaks["f64"]["probe"] = 20e12
    r = bench.roofline_of(pm, pm.J7_VAR, "f64", n, res, peaks, 6788.6)
    assert r["bound"] == "hbm" and abs(r["frac"] - 72 * lups / 1e9 / 6788.6) < 1e-12


def test_tuner_candidates_cover_every_kernel_family():
    from paper_1410_3060_gb300 import tune
    c = tune.default_candidates(None)
    assert set(v for b, s, v in c if b == 1) == set(range(1, 18))
    for b in (2, 3, 4):
        fams = {(s, v) for bb, s, v in c if bb == b}
        assert {(3, 10), (3, 11), (3, 12), (3, 17), (1, 0), (2, 0)} <= fams


def test_reference_arm_prints_one_contract_line():
    """bench.py --impl reference runs on the host cores (the FP64 oracle) and
    prints one JSON line with the contract's keys."""
    import json
    import subprocess
    import sys
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--n", "24",
                          "--T", "2", "--steps", "1", "--warmup", "1"], capture_output=True, text=True, timeout=600,
                         cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "dtype", "config", "e2e", "cpu_baseline", "impl"):
        assert k in d, k
    assert d["impl"] == "reference" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1


def test_traffic_is_per_launch(bench):
    """A profiled configuration's DRAM traffic is per launch: bytes per update
    x the n^3 x levels updates of one pass (3 levels of the 7-point constant
    FP32 wavefront: 2.53 B x 3 n^3, close to its 8 algorithmic bytes per
    point and pass)."""
    n = 512
    rec = {}
    bench.add_traffic(rec, "j7_const", "f32", {"time_block": 3, "variant": 12}, n)
    assert abs(rec["traffic"] - 2.53 * 3 * n ** 3) < 1.0
    assert abs(rec["traffic"] / n ** 3 - 8.0) < 0.5
    assert bench.adjoint_bytes_per_lup(2, 4, 2) == 18.0 and bench.adjoint_bytes_per_lup(2, 4, 1) == 36.0
    assert bench.adjoint_bytes_per_lup(1, 4, 2) == 4.0


def test_fwd_adj_j7_bytes(bench):
    """7-point variable forward + backward, FP32, passes of 2 levels, T = 64,
    K = 16, gradient batch 16: forward 18 B, recompute of 3 of 4 segments
    20 B x 0.75, adjoint 20 B, gradient reads 8 B and 7 FP64 arrays read and
    written once per 16 steps (7 B)."""
    assert abs(bench.fwd_adj_j7_bytes_per_lup(4, 64, 16, 16, 2) - (18 + 15 + 20 + 8 + 7)) < 1e-12
    assert abs(bench.fwd_adj_j7_bytes_per_lup(4, 64, 16, 16, 1) - (36 + 27 + 36 + 8 + 7)) < 1e-12
