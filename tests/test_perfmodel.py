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
