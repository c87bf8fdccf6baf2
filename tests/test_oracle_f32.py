"""Pins of the oracle's FP32 evaluation (oracle_f32.c), the definition of the
FP32 mode: fields and coefficients stored in FP32, FP32 arithmetic, the same
naive sweep of Fig. 1 (Sect. 3.1).

* On dyadic inputs whose every intermediate value fits a float exactly
  (weights and data on coarse binary grids, few steps), the FP32 evaluation
  equals the pinned FP64 oracle bit for bit.  A dropped or extra term, a
  wrong offset, sign, axis or coefficient index breaks that equality.
* On the benchmarks' random inputs its difference from the FP64 oracle is
  nonzero and of the size of FP32 rounding (it really runs in FP32).
"""
import numpy as np
import pytest

import oracle
from oracle import J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA
from paper_1410_3060_gb300 import workloads as wl

ALL_KINDS = [J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA]
EPS32 = 2.0 ** -24


def dyadic_case(kind, n, rng):
    """Inputs on binary grids: data k/4 in [-2, 2], coefficients k/16."""
    R = oracle.RADIUS[kind]
    nx, ny, nz = n

    def field():
        a = np.zeros(wl.padded_shape(n, R))
        a[R:R + nz, R:R + ny, R:R + nx] = rng.integers(-8, 9, size=(nz, ny, nx)) / 4.0
        return a

    W = None
    if oracle.NUM_ARRAYS[kind]:
        W = np.zeros((oracle.NUM_ARRAYS[kind],) + wl.padded_shape(n, R))
        lo = 0 if kind in (J7_VAR, W25_ALPHA) else -2
        for k in range(W.shape[0]):
            W[k, R:R + nz, R:R + ny, R:R + nx] = rng.integers(lo, 3, size=(nz, ny, nx)) / 16.0
    w = {J7_CONST: [0.5, 0.0625], W25_CONST: [0.125, -3.0, 0.5, -0.25, 0.125, -0.0625],
         W25_ALPHA: [-3.0, 0.5, -0.25, 0.125, -0.0625]}.get(kind)
    T = 3 if R == 1 else 2
    return field(), field(), w, W, T


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_f32_equals_fp64_oracle_on_dyadic_inputs(kind):
    rng = np.random.default_rng(30 + kind)
    up, u, w, W, T = dyadic_case(kind, (10, 9, 8), rng)
    rz = 3
    p64, u64, tr64 = oracle.forward(kind, up, u, w, W, T, rcv_z=rz)
    p32, u32, tr32 = oracle.forward_f32(kind, up, u, w, W, T, rcv_z=rz)
    # a nontrivial result on a fine binary grid (the steps really mixed terms)
    assert np.abs(u64).max() > 0 and np.any(u64 * 2 ** 8 != np.round(u64 * 2 ** 8))
    np.testing.assert_array_equal(u32, u64)
    np.testing.assert_array_equal(p32, p64)
    np.testing.assert_array_equal(tr32, tr64)


@pytest.mark.parametrize("kind", ALL_KINDS)
def test_f32_error_is_float_rounding_sized(kind):
    """Random inputs of the benchmarks' distributions: 0 < error <= a priori
    FP32 bound (inputs rounded once, then per step at most terms + 2
    roundings; the wave kinds' error may grow by a further factor T)."""
    T = 5
    wk = wl.make(kind, (14, 12, 11), T, seed=4)
    _, u64, _ = oracle.forward(kind, wk.u_prev, wk.u, wk.w, wk.W, T)
    _, u32, _ = oracle.forward_f32(kind, wk.u_prev, wk.u, wk.w, wk.W, T)
    err = np.abs(u32 - u64).max() / np.abs(u64).max()
    terms = 6 * wk.R + 3
    bound = 4.0 * (T + 1) * terms * EPS32 * ((T + 1) if oracle.SECOND_ORDER[kind] else 1)
    assert 0 < err <= bound, (err, bound)
    # the result is representable in float (float storage)
    np.testing.assert_array_equal(u32, u32.astype(np.float32).astype(np.float64))


def test_f32_threads_do_not_change_bits():
    wk = wl.make(W25_VAR, 18, 3, seed=1)
    a = oracle.forward_f32(W25_VAR, wk.u_prev, wk.u, None, wk.W, 3, threads=1)[1]
    b = oracle.forward_f32(W25_VAR, wk.u_prev, wk.u, None, wk.W, 3, threads=4)[1]
    np.testing.assert_array_equal(a, b)
