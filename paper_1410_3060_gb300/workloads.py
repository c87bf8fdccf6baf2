"""Seeded synthetic inputs for the stencil workloads.

This module is shared by the CUDA path's tests and benchmark and by the CPU
oracle; it holds no stencil arithmetic -- only the input recipes.  All
values are generated in FP64 with ``numpy.random.default_rng`` (PCG64), one
sub-stream per array (``seed * 100 + array_id``); FP32 runs cast these FP64
inputs.  Arrays are halo-padded C-order (nz+2R, ny+2R, nx+2R) with a zero
halo (the interior is 1..N in every axis, paper Sect. 3.1 / Fig. 1).

Workloads (paper Fig. 1 operators; sizes, weights and distributions are
those of the benchmark configurations):

* ``j7_const``  -- 7-point constant, u' = 0.4 u + 0.1 (sum of 6 faces),
  u0 ~ U[-1, 1]  (Fig. 1b).
* ``j7_var``    -- 7-point variable, 7 arrays ~ U[0, 0.14], u0 ~ U[-1, 1]
  (Fig. 1c).
* ``w25_const`` -- 25-point wave, alpha = 0.1, 8th-order Laplacian weights
  per axis (-205/72, 8/5, -1/5, 8/315, -1/560); the 3D centre weight is the
  sum of the three per-axis centres, 3 * (-205/72).  u0 = u(-1) = unit
  Gaussian pulse (sigma 8 cells) at the centre plus 1e-3 * U[-1, 1] noise
  (Fig. 1e with scalar alpha).
* ``w25_var``   -- 25-point wave with 13 arrays (Fig. 1d ordering: index 0
  centre, 3(r-1)+a+1 for axis a in {x, y, z} and radius r):
  c_{a,r} = w_r * v * (1 + 0.1 xi_{a,r}), xi ~ U[-1, 1], v a smooth field in
  [0.05, 0.12] (periodic Gaussian filter, sigma 16 cells, of N(0,1) noise,
  min-max mapped), c0 = -2 * sum_{a,r} c_{a,r} so that constants are
  preserved.
* ``j25_var``   -- Fig. 1d first order in time: 13 arrays, W_{a,r} ~
  U[0, 0.02], W0 = 1 - 2 sum W_{a,r} (weights sum to one).
* ``w25_alpha`` -- Fig. 1e with a domain-sized alpha ~ U[0.05, 0.12].
* ``fwi``       -- the differentiable 25-point variable wave workload:
  pulse (sigma 8) at (N/2, N/2, 24), receivers on interior plane z = 8,
  observed data from v_true = v * (1 + 0.05 exp(-|x - x_b|^2 / (2 * 8^2)))
  with x_b = (N/2, N/2, 40); a 48^3 copy scales these to sigma 3 at
  (24, 24, 12), receivers z = 4, blob sigma 4 at (24, 24, 24).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# kind numbers (same numbering as the C interface)
J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA = 1, 2, 3, 4, 5, 6
RADIUS = {J7_CONST: 1, J7_VAR: 1, W25_CONST: 4, W25_VAR: 4, J25_VAR: 4, W25_ALPHA: 4}
KIND_NAMES = {J7_CONST: "j7_const", J7_VAR: "j7_var", W25_CONST: "w25_const",
              W25_VAR: "w25_var", J25_VAR: "j25_var", W25_ALPHA: "w25_alpha"}

# 8th-order central second-derivative weights, per axis (centre, r = 1..4)
L8_1D = (-205.0 / 72.0, 8.0 / 5.0, -1.0 / 5.0, 8.0 / 315.0, -1.0 / 560.0)


@dataclass
class Workload:
    kind: int
    n: tuple            # (nx, ny, nz) interior
    T: int
    u_prev: np.ndarray  # padded FP64
    u: np.ndarray       # padded FP64
    w: np.ndarray | None = None      # host scalars
    W: np.ndarray | None = None      # (k, pz, py, px) FP64
    meta: dict = field(default_factory=dict)

    @property
    def R(self):
        return RADIUS[self.kind]


def _rng(seed: int, array_id: int) -> np.random.Generator:
    return np.random.default_rng(seed * 100 + array_id)


def padded_shape(n, R):
    nx, ny, nz = n
    return (nz + 2 * R, ny + 2 * R, nx + 2 * R)


def interior_view(a, R):
    return a[..., R:-R, R:-R, R:-R]


def _padded_uniform(n, R, lo, hi, rng):
    a = np.zeros(padded_shape(n, R))
    nx, ny, nz = n
    a[R:R + nz, R:R + ny, R:R + nx] = rng.uniform(lo, hi, size=(nz, ny, nx))
    return a


def _as_n(n):
    return (n, n, n) if np.isscalar(n) else tuple(int(v) for v in n)


def gaussian_pulse(n, R, centre, sigma):
    """exp(-|x - c|^2 / (2 sigma^2)) on the interior (zero-based interior
    coordinates, peak 1 at ``centre`` = (x, y, z)), zero halo."""
    nx, ny, nz = n
    cx, cy, cz = centre
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    g = np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2.0 * sigma * sigma))
    a = np.zeros(padded_shape(n, R))
    a[R:R + nz, R:R + ny, R:R + nx] = g
    return a


def smooth_field(n, sigma, lo, hi, rng):
    """N(0,1) noise filtered by a periodic Gaussian (FFT, std ``sigma`` cells)
    and min-max mapped to [lo, hi]; interior shape (nz, ny, nx)."""
    nx, ny, nz = n
    noise = rng.standard_normal((nz, ny, nx))
    kz = np.fft.fftfreq(nz)[:, None, None]
    ky = np.fft.fftfreq(ny)[None, :, None]
    kx = np.fft.rfftfreq(nx)[None, None, :]
    filt = np.exp(-2.0 * (np.pi * sigma) ** 2 * (kx ** 2 + ky ** 2 + kz ** 2))
    f = np.fft.irfftn(np.fft.rfftn(noise) * filt, s=(nz, ny, nx), axes=(0, 1, 2))
    fmin, fmax = f.min(), f.max()
    return lo + (hi - lo) * (f - fmin) / (fmax - fmin)


def j7_const(n=64, T=8, seed=0):
    n = _as_n(n)
    R = 1
    u = _padded_uniform(n, R, -1.0, 1.0, _rng(seed, 0))
    return Workload(J7_CONST, n, T, u.copy(), u, w=np.array([0.4, 0.1]),
                    meta={"u0": "U[-1,1]", "w": [0.4, 0.1], "seed": seed})


def j7_var(n=512, T=64, seed=0):
    n = _as_n(n)
    R = 1
    u = _padded_uniform(n, R, -1.0, 1.0, _rng(seed, 0))
    W = np.zeros((7,) + padded_shape(n, R))
    for k in range(7):
        nx, ny, nz = n
        W[k, R:R + nz, R:R + ny, R:R + nx] = _rng(seed, 1 + k).uniform(0.0, 0.14, size=(nz, ny, nx))
    return Workload(J7_VAR, n, T, u.copy(), u, W=W,
                    meta={"u0": "U[-1,1]", "W": "U[0,0.14]", "seed": seed})


def w25_const_weights(alpha=0.1):
    return np.array([alpha, 3.0 * L8_1D[0], L8_1D[1], L8_1D[2], L8_1D[3], L8_1D[4]])


def w25_const(n=512, T=100, seed=0, alpha=0.1, sigma=8.0):
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    u = gaussian_pulse(n, R, (nx // 2, ny // 2, nz // 2), sigma)
    u[R:R + nz, R:R + ny, R:R + nx] += 1e-3 * _rng(seed, 0).uniform(-1.0, 1.0, size=(nz, ny, nx))
    return Workload(W25_CONST, n, T, u.copy(), u, w=w25_const_weights(alpha),
                    meta={"u0": f"pulse sigma={sigma} at centre + 1e-3 U[-1,1]", "alpha": alpha,
                          "seed": seed})


def w25_var_coeffs(n, v, seed, xi_amp=0.1):
    """13 arrays from the smooth field v (interior shape): c_{a,r} = w_r v (1 + xi_amp xi),
    c0 = -2 sum c_{a,r}."""
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    W = np.zeros((13,) + padded_shape(n, R))
    c0 = np.zeros((nz, ny, nx))
    for r in range(1, 5):
        for a in range(3):
            k = 3 * (r - 1) + a + 1
            xi = _rng(seed, 10 + k).uniform(-1.0, 1.0, size=(nz, ny, nx))
            c = L8_1D[r] * v * (1.0 + xi_amp * xi)
            W[k, R:R + nz, R:R + ny, R:R + nx] = c
            c0 -= 2.0 * c
    W[0, R:R + nz, R:R + ny, R:R + nx] = c0
    return W


def w25_var(n=512, T=64, seed=0, sigma_v=16.0, vlo=0.05, vhi=0.12):
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    v = smooth_field(n, sigma_v, vlo, vhi, _rng(seed, 5))
    W = w25_var_coeffs(n, v, seed)
    u = gaussian_pulse(n, R, (nx // 2, ny // 2, nz // 2), 8.0)
    u[R:R + nz, R:R + ny, R:R + nx] += 1e-3 * _rng(seed, 0).uniform(-1.0, 1.0, size=(nz, ny, nx))
    return Workload(W25_VAR, n, T, u.copy(), u, W=W,
                    meta={"u0": "pulse sigma=8 at centre + 1e-3 U[-1,1]",
                          "v": f"gauss-filtered sigma={sigma_v} in [{vlo},{vhi}]",
                          "c0": "-2*sum(c_ar)", "seed": seed})


def j25_var(n=128, T=16, seed=0):
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    W = np.zeros((13,) + padded_shape(n, R))
    s = np.zeros((nz, ny, nx))
    for k in range(1, 13):
        c = _rng(seed, 10 + k).uniform(0.0, 0.02, size=(nz, ny, nx))
        W[k, R:R + nz, R:R + ny, R:R + nx] = c
        s += 2.0 * c
    W[0, R:R + nz, R:R + ny, R:R + nx] = 1.0 - s
    u = _padded_uniform(n, R, -1.0, 1.0, _rng(seed, 0))
    return Workload(J25_VAR, n, T, u.copy(), u, W=W,
                    meta={"u0": "U[-1,1]", "W": "U[0,0.02], W0=1-2sum", "seed": seed})


def w25_alpha(n=128, T=16, seed=0):
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    A = np.zeros((1,) + padded_shape(n, R))
    A[0, R:R + nz, R:R + ny, R:R + nx] = _rng(seed, 1).uniform(0.05, 0.12, size=(nz, ny, nx))
    u = gaussian_pulse(n, R, (nx // 2, ny // 2, nz // 2), 8.0)
    u[R:R + nz, R:R + ny, R:R + nx] += 1e-3 * _rng(seed, 0).uniform(-1.0, 1.0, size=(nz, ny, nx))
    w = np.array([3.0 * L8_1D[0], L8_1D[1], L8_1D[2], L8_1D[3], L8_1D[4]])
    return Workload(W25_ALPHA, n, T, u.copy(), u, w=w, W=A,
                    meta={"u0": "pulse sigma=8 + 1e-3 U[-1,1]", "alpha": "U[0.05,0.12]", "seed": seed})


@dataclass
class FwiWorkload:
    n: tuple
    T: int
    K: int
    rcv_z: int
    u0: np.ndarray        # padded FP64
    W: np.ndarray         # model coefficients (13, ...) FP64
    W_true: np.ndarray    # coefficients that generate the observed data
    meta: dict = field(default_factory=dict)
    R: int = 4
    kind: int = W25_VAR


def fwi(n=256, T=200, K=20, seed=0):
    """Differentiable wave workload.  The observed data d are produced by a
    forward run with ``W_true`` (done by the caller: the oracle in tests)."""
    n = _as_n(n)
    R = 4
    nx, ny, nz = n
    if nx == 48:
        pulse_c, pulse_s, rcv_z, blob_c, blob_s = (24, 24, 12), 3.0, 4, (24, 24, 24), 4.0
    else:
        pulse_c, pulse_s, rcv_z, blob_c, blob_s = (nx // 2, ny // 2, 24), 8.0, 8, (nx // 2, ny // 2, 40), 8.0
    rng_v = _rng(seed, 5)
    v = smooth_field(n, 16.0, 0.05, 0.12, rng_v)
    z = np.arange(nz)[:, None, None]
    y = np.arange(ny)[None, :, None]
    x = np.arange(nx)[None, None, :]
    blob = np.exp(-((x - blob_c[0]) ** 2 + (y - blob_c[1]) ** 2 + (z - blob_c[2]) ** 2)
                  / (2.0 * blob_s * blob_s))
    v_true = v * (1.0 + 0.05 * blob)
    W = w25_var_coeffs(n, v, seed)
    W_true = w25_var_coeffs(n, v_true, seed)
    u0 = gaussian_pulse(n, R, pulse_c, pulse_s)
    u0[R:R + nz, R:R + ny, R:R + nx] += 1e-3 * _rng(seed, 0).uniform(-1.0, 1.0, size=(nz, ny, nx))
    return FwiWorkload(n, T, K, rcv_z, u0, W, W_true,
                       meta={"pulse": [list(pulse_c), pulse_s], "rcv_z": rcv_z,
                             "blob": [list(blob_c), blob_s, 0.05], "seed": seed})


def make(kind, n, T, seed=0):
    """Workload of the given kind at interior size n with the standard recipe."""
    if kind == J7_CONST:
        return j7_const(n, T, seed)
    if kind == J7_VAR:
        return j7_var(n, T, seed)
    if kind == W25_CONST:
        return w25_const(n, T, seed, sigma=min(8.0, max(1.0, _as_n(n)[0] / 8.0)))
    if kind == W25_VAR:
        return w25_var(n, T, seed, sigma_v=min(16.0, max(2.0, _as_n(n)[0] / 8.0)))
    if kind == J25_VAR:
        return j25_var(n, T, seed)
    if kind == W25_ALPHA:
        return w25_alpha(n, T, seed)
    raise ValueError(f"unknown kind {kind}")
