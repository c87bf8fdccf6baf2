"""The paper's printed model numbers (tests/golden/paper_model_numbers.json)
pin the code-balance, roofline and cache-block helpers."""
import json
import os

import pytest

from paper_1410_3060_gb300 import perfmodel as pm

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_model_numbers.json")))


@pytest.mark.parametrize("e", GOLD["code_balance_fp64"])
def test_cpu_code_balance(e):
    assert pm.cpu_code_balance(e["kind"], 8, e["write_allocate"]) == e["bytes_per_lup"]


@pytest.mark.parametrize("e", GOLD["roofline_gluops"])
def test_roofline(e):
    assert round(pm.roofline(e["bandwidth_gbs"] * 1e9, e["bytes_per_lup"]) / 1e9, 2) == e["glups"]


@pytest.mark.parametrize("e", GOLD["cache_block"])
def test_cache_block(e):
    assert pm.cache_block_bytes(e["Dw"], e["NF"], 1.0, e["ND"], e["R"]) == e["bytes_per_Nxb"]


@pytest.mark.parametrize("e", GOLD["wavefront_width"])
def test_wavefront_width(e):
    assert pm.wavefront_width(e["Dw"], e["NF"], e["R"]) == e["Ww"]


def test_general_R_formula_reduces_to_R1_form():
    for Dw in (4, 8, 12):
        for NF in (0, 1, 3):
            Ww = Dw + NF - 1
            r1 = Dw * Dw / 2 + Dw * NF + 2 * (Dw + Ww)
            assert pm.cache_block_bytes(Dw, NF, 1.0, 1, 1) == r1


def test_gpu_bytes():
    # no write-allocate on the GPU: FP64 7pt const 16, 7pt var 72, 25pt wave 24, 25pt var wave 128
    assert [pm.gpu_bytes_per_lup(k, 8) for k in (1, 2, 3, 4)] == [16, 72, 24, 128]
    assert [pm.gpu_bytes_per_lup(k, 4) for k in (1, 2, 3, 4)] == [8, 36, 12, 64]


# ---- GPU block model (the counterpart of the Sect. 5.3 cache block)

PROFILED = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "profiled_smem.json")))


@pytest.fixture(scope="module")
def st():
    from paper_1410_3060_gb300 import build, stencil
    build.build()
    return stencil


def _configs():
    for kind in (1, 2):
        for dtype, word in ((1, 4), (0, 8)):
            for B in (1, 2, 3, 4):
                for v in (0, 10, 11, 12, 17):
                    yield ("wf", kind, dtype, word, B, v)
    for kind in (1, 2, 3, 4, 5, 6):
        for dtype, word in ((1, 4), (0, 8)):
            for v in (13, 14, 15, 16):
                yield ("vec", kind, dtype, word, 1, v)


def test_block_model_reproduces_every_kernel_configuration(st):
    """The model's shared memory, threads and tile extents equal the kernels'
    own launch constants (stencil_pass_info) for every configuration the
    library serves."""
    n = 0
    for fam, kind, dtype, word, B, v in _configs():
        ref = st.pass_info(kind, dtype, B, 3 if fam == "wf" else 0, v)
        if ref is None:
            continue
        m = pm.wavefront_block(kind, word, B, v) if fam == "wf" else pm.vector_sweep_block(kind, word, v)
        assert (m["smem_bytes"], m["threads"], tuple(m["computed"]), tuple(m["owned"])) == (
            ref["smem_bytes"], ref["threads"], ref["computed"], ref["owned"]), (fam, kind, dtype, B, v)
        n += 1
    assert n >= 60


@pytest.mark.parametrize("e", PROFILED["entries"])
def test_block_model_reproduces_profiled_shared_memory(e):
    """Against ncu's launch__shared_mem_per_block_dynamic of profiled launches."""
    word = 4 if e["dtype"] == 1 else 8
    if e["family"] == "wavefront":
        m = pm.wavefront_block(e["kind"], word, e["levels"], e["variant"])
    elif e["family"] == "vector":
        m = pm.vector_sweep_block(e["kind"], word, e["variant"])
    else:
        m = pm.two_level_block(e["kind"])
    assert m["smem_bytes"] == e["smem_bytes"]


def test_two_level_model_matches_library(st):
    for kind in (3, 4, 5):
        ref = st.pass_info(kind, 1, 2, 4, 0)
        m = pm.two_level_block(kind)
        assert (m["smem_bytes"], m["threads"], tuple(m["computed"]), tuple(m["owned"])) == (
            ref["smem_bytes"], ref["threads"], ref["computed"], ref["owned"])
    assert st.pass_info(4, 0, 2, 4, 0) is None       # FP32 only


def test_block_model_limits():
    """Depth-4 7-point variable tiles: the coefficient ring of 3 planes x 7
    arrays does not fit beside the other buffers (levels above 1 read their
    coefficients from L2); the ring's register lower bound grows with the
    depth and every served tile fits the 128 registers a 512-thread CTA
    allows; the overlapped halo makes deeper passes more redundant."""
    m4 = pm.wavefront_block(2, 4, 4, 11)
    assert not m4["coef_ring"] and m4["fits"]
    assert pm.wavefront_block(2, 4, 2, 11)["coef_ring"]
    assert [pm.wavefront_block(1, 4, B, 12)["regs_min"] for B in (1, 2, 3)] == [48, 72, 96]
    assert pm.wavefront_block(1, 4, 3, 12)["regs_cap"] == 128
    red = [pm.wavefront_block(1, 4, B, 12)["redundancy"] for B in (1, 2, 3)]
    assert red[0] < red[1] < red[2]
    # a 64 x 64 tile at depth 4 would need 4 x 3 x 8 + 8 + 16 = 120 of 128
    # registers for its rings alone: the library serves depth 4 with 2 rows
    # per thread instead
    assert pm.wavefront_tile(12, 4) == (2, 2, 16)


def test_tuner_candidates_follow_the_model():
    """Candidates are the model's feasible configurations in modelled HBM
    byte order; the 7-point FP32 list starts with the deepest register
    wavefront passes and the one-level tiles come last."""
    from paper_1410_3060_gb300 import tune
    c = tune.model_candidates(1, 1)
    bytes_ = [m["dram_bytes_per_lup"] for _, _, _, m in c]
    assert bytes_ == sorted(bytes_)
    assert c[0][0] == 4 and c[0][1] == 3 and all(m["fits"] for *_, m in c)
    assert c[-1][0] == 1
    # FP32 7-point rows are not 16-byte aligned: no vectorised 16-byte
    # tiles; the wavefront's 4-point rows (8-byte halves) are candidates
    assert not any(13 <= v <= 16 for _, _, v, _ in c)
    assert {v for _, _, v, _ in c if v >= 17} == {17}
    assert not any(v >= 17 for _, _, v, _ in tune.model_candidates(1, 0))
    c25 = tune.model_candidates(4, 1)
    assert {v for _, _, v, _ in c25 if v >= 13} == {13, 14, 15, 16}


def test_two_level_candidates():
    """The two-level pass (scheme 4, depth 2) is a candidate for the FP32
    13-array kinds and the constant wave, modelled at half the plain bytes
    per update, and for no FP64 plan or other kind."""
    from paper_1410_3060_gb300 import tune
    for kind in (3, 4, 5):
        c = [x for x in tune.model_candidates(kind, 1) if x[1] == 4]
        assert [(b, v) for b, _, v, _ in c] == [(2, 0)]
        assert c[0][3]["dram_bytes_per_lup"] == pm.dram_bytes_per_lup(kind, 4, 2)
        assert not any(x[1] == 4 for x in tune.model_candidates(kind, 0))
    for kind in (1, 2, 6):
        assert not any(x[1] == 4 for x in tune.model_candidates(kind, 1))
    # the constant wave keeps two planes in flight: its rings are larger
    assert pm.two_level_block(3)["smem_bytes"] > pm.two_level_block(4)["smem_bytes"]
