"""Plant plausible mistakes in a copy of the oracle source and check that the
pins catch each one (the pins must not pass a wrong oracle).

Each mutation replaces one expression of ``oracle.c`` in a temporary copy,
compiles it with the oracle's flags, and re-runs one pin against it.
"""
import numpy as np
import pytest

import oracle
from oracle import oracle as ora
import test_oracle_pins as pins

MUTATIONS = {
    # sign of the previous time level in the scalar-alpha wave update (Fig. 1e)
    "wave_prev_sign": ("return 2.0 * c[i] - p[i] + w[0] * s;", "return 2.0 * c[i] + p[i] + w[0] * s;"),
    # x+1 neighbour read at x-1 for W2 (Fig. 1c)
    "j7var_offset": ("+ W[2 * n + i] * c[i + sx]", "+ W[2 * n + i] * c[i - sx]"),
    # z-pair dropped from the 7-point constant stencil (Fig. 1b)
    "j7_drop_z": ("+ w[1] * (c[i - sz] + c[i + sz]);", ";"),
    # axes of the Fig. 1d coefficient index swapped (x <-> z)
    "w25var_axis": ("s += W[(int64_t)(3 * (r - 1) + a + 1) * n + i] * (c[i - st] + c[i + st]);",
                    "s += W[(int64_t)(3 * (r - 1) + (2 - a) + 1) * n + i] * (c[i - st] + c[i + st]);"),
    # adjoint: lam^{n+2} term dropped from the second-order recursion
    "adjoint_drop_l2": ("if (so) v = 2.0 * l1[i] + v - l2[i];", "if (so) v = 2.0 * l1[i] + v;"),
    # adjoint: coefficient gathered at the target instead of the source point
    "adjoint_gather_target": ("s += W[k * n + src] * y[src];", "s += W[k * n + q] * y[src];"),
    # gradient: neighbour pair replaced by twice the centre
    "grad_pair": ("grad[(int64_t)(3 * (r - 1) + a + 1) * n + i] += l * (u[i - st] + u[i + st]);",
                  "grad[(int64_t)(3 * (r - 1) + a + 1) * n + i] += l * (u[i] + u[i]);"),
}


def run_pin(name):
    if name == "wave_prev_sign":
        pins.test_w25_const_leapfrog_eigenmode((3, 1, 5))
    elif name in ("j7var_offset",):
        pins.test_impulse_response_matches_offset_table(oracle.J7_VAR)
    elif name == "j7_drop_z":
        pins.test_j7_sine_eigenmode((6, 6, 6), (1, 2, 3))
    elif name == "w25var_axis":
        pins.test_impulse_response_matches_offset_table(oracle.W25_VAR)
    elif name == "adjoint_drop_l2":
        pins.test_adjoint_dot_product(oracle.W25_VAR, 4)
    elif name == "adjoint_gather_target":
        pins.test_adjoint_dot_product(oracle.J25_VAR, 1)
    elif name == "grad_pair":
        pins.test_gradient_finite_differences_small(oracle.W25_VAR)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_pin_catches_mutation(name, tmp_path):
    old, new = MUTATIONS[name]
    src = ora.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    run_pin(name)  # the real oracle passes
    path = ora.compile_variant(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    with ora.swapped_library(path):
        with pytest.raises(AssertionError):
            run_pin(name)


# ---- the FP32 evaluation (oracle_f32.c): mistakes planted there must break
# its bit-for-bit agreement with the FP64 oracle on dyadic inputs
MUTATIONS_F32 = {
    # z pair dropped from the 7-point constant stencil
    "f32_j7_drop_z": ("+ lam[1] * (u[i - g->sz] + u[i + g->sz]);", ";"),
    # sign of the previous level in the wave update
    "f32_wave_prev_sign": ("return 2.0f * u[i] - up[i] + al * acc;", "return 2.0f * u[i] + up[i] + al * acc;"),
    # y-1 neighbour of the 7-point variable stencil read at y+1
    "f32_j7var_offset": ("+ A[3 * n + i] * u[i - g->sy]", "+ A[3 * n + i] * u[i + g->sy]"),
    # coefficient of the radius-r pair taken from radius r - 1's arrays
    "f32_w25var_radius": ("acc += A[(int64_t)(3 * (r - 1) + a + 1) * n + i] * (u[i - d] + u[i + d]);",
                          "acc += A[(int64_t)(3 * (r > 1 ? r - 2 : 0) + a + 1) * n + i] * (u[i - d] + u[i + d]);"),
}
F32_PIN_KIND = {"f32_j7_drop_z": oracle.J7_CONST, "f32_wave_prev_sign": oracle.W25_CONST,
                "f32_j7var_offset": oracle.J7_VAR, "f32_w25var_radius": oracle.W25_VAR}


@pytest.mark.parametrize("name", sorted(MUTATIONS_F32))
def test_f32_pin_catches_mutation(name, tmp_path):
    import test_oracle_f32 as pins32
    old, new = MUTATIONS_F32[name]
    src = ora.source_text_f32()
    assert src.count(old) == 1, f"mutation anchor not unique: {old}"
    kind = F32_PIN_KIND[name]
    pins32.test_f32_equals_fp64_oracle_on_dyadic_inputs(kind)   # the real FP32 evaluation passes
    path = ora.compile_variant_f32(src.replace(old, new), str(tmp_path / f"lib_{name}.so"))
    with ora.swapped_library(path):
        with pytest.raises(AssertionError):
            pins32.test_f32_equals_fp64_oracle_on_dyadic_inputs(kind)
