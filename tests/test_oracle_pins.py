"""Pins of the CPU oracle against what the paper and the mathematics fix.

None of these re-types the oracle's update formula: each checks a property
that a dropped term, a wrong sign, a wrong offset or a transposed operand
breaks -- invariants (constant preservation, discrete energy), closed forms
(Dirichlet sine eigenmodes, the eigenpairs of the truncated 1D Toeplitz
operator from a library eigensolver), brute force on tiny inputs (impulse
responses against the offset table of Fig. 1, exact rational Laurent
coefficients), symmetries, and the transposition identity and finite
differences for the adjoint.
"""
import itertools
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA
from paper_1410_3060_gb300 import workloads as wl

EPS = np.finfo(np.float64).eps
ALL_KINDS = [J7_CONST, J7_VAR, W25_CONST, W25_VAR, J25_VAR, W25_ALPHA]
VAR_KINDS = [J7_VAR, W25_VAR, J25_VAR, W25_ALPHA]

# Fig. 1 offset table, written out independently of the oracle:
# (array index k, (dx, dy, dz)) for every term of the operator.
OFFSETS_J7_VAR = [(0, (0, 0, 0)), (1, (-1, 0, 0)), (2, (1, 0, 0)), (3, (0, -1, 0)),
                  (4, (0, 1, 0)), (5, (0, 0, -1)), (6, (0, 0, 1))]


def offsets_25():
    out = [(0, (0, 0, 0))]
    for r in range(1, 5):
        for a, e in enumerate([(1, 0, 0), (0, 1, 0), (0, 0, 1)]):
            k = 3 * (r - 1) + a + 1
            out.append((k, tuple(r * v for v in e)))
            out.append((k, tuple(-r * v for v in e)))
    return out


def rand_interior(n, R, rng, lo=-1.0, hi=1.0):
    nx, ny, nz = n
    a = np.zeros(wl.padded_shape(n, R))
    a[R:R + nz, R:R + ny, R:R + nx] = rng.uniform(lo, hi, size=(nz, ny, nx))
    return a


def rand_coeffs(kind, n, rng, lo=0.1, hi=1.0):
    R = oracle.RADIUS[kind]
    k = oracle.NUM_ARRAYS[kind]
    W = np.zeros((k,) + wl.padded_shape(n, R))
    for i in range(k):
        W[i] = rand_interior(n, R, rng, lo, hi)
    return W


def default_weights(kind):
    if kind == J7_CONST:
        return np.array([0.4, 0.1])
    if kind == W25_CONST:
        return wl.w25_const_weights(0.1)
    if kind == W25_ALPHA:
        return wl.w25_const_weights(0.1)[1:]
    return None


# ---------------------------------------------------------------- P1 constants
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_constant_field_preserved(kind):
    """Weights that sum to one (first order) or an operator that annihilates
    constants (wave kinds: w0 + 2 sum w_r = 0) keep a constant field, halo
    included, constant (Sect. 3.1 update definitions)."""
    rng = np.random.default_rng(1)
    n = (11, 10, 12)
    R = oracle.RADIUS[kind]
    c = 0.7
    u = np.full(wl.padded_shape(n, R), c)
    w, W = default_weights(kind), None
    if kind == J7_VAR:
        W = rng.uniform(0.1, 1.0, size=(7,) + u.shape)
        W /= W.sum(axis=0, keepdims=True)
    elif kind == W25_VAR:
        v = rng.uniform(0.05, 0.12, size=(n[2], n[1], n[0]))
        W = wl.w25_var_coeffs(n, v, seed=3)
    elif kind == J25_VAR:
        W = wl.j25_var(n, 1, seed=2).W
    elif kind == W25_ALPHA:
        W = rng.uniform(0.05, 0.12, size=(1,) + u.shape)
    T = 7
    p, q, _ = oracle.forward(kind, u, u, w, W, T)
    assert np.max(np.abs(q - c)) <= 64 * T * EPS
    assert np.max(np.abs(p - c)) <= 64 * T * EPS


def test_w25_weights_annihilate_constants_exactly():
    """The 8th-order weights satisfy w0 + 2(w1 + w2 + w3 + w4) = 0 in rationals."""
    w = [Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560)]
    assert w[0] + 2 * sum(w[1:]) == 0
    assert np.allclose(wl.L8_1D, [float(x) for x in w], rtol=0, atol=0)


# ---------------------------------------------------------------- P2 sine modes
@pytest.mark.parametrize("n,k", [((6, 6, 6), (1, 2, 3)), ((9, 7, 8), (2, 1, 5)),
                                 ((16, 16, 16), (3, 7, 1))])
def test_j7_sine_eigenmode(n, k):
    """On a zero Dirichlet halo, phi = prod_a sin(pi k_a i_a / (N_a + 1))
    (i_a = 1..N_a) is an eigenvector of Fig. 1b with eigenvalue
    w1 + 2 w2 sum_a cos(pi k_a / (N_a + 1))."""
    R = 1
    w1, w2 = 0.4, 0.1
    nx, ny, nz = n
    phi = np.zeros(wl.padded_shape(n, R))
    ix = np.sin(np.pi * k[0] * np.arange(1, nx + 1) / (nx + 1))
    iy = np.sin(np.pi * k[1] * np.arange(1, ny + 1) / (ny + 1))
    iz = np.sin(np.pi * k[2] * np.arange(1, nz + 1) / (nz + 1))
    phi[1:-1, 1:-1, 1:-1] = iz[:, None, None] * iy[None, :, None] * ix[None, None, :]
    mu = w1 + 2 * w2 * (np.cos(np.pi * k[0] / (nx + 1)) + np.cos(np.pi * k[1] / (ny + 1))
                        + np.cos(np.pi * k[2] / (nz + 1)))
    T = 9
    p, u, _ = oracle.forward(J7_CONST, phi, phi, [w1, w2], None, T)
    assert np.max(np.abs(u - mu ** T * phi)) <= 1e-14
    assert np.max(np.abs(p - mu ** (T - 1) * phi)) <= 1e-14


def test_j7_var_constant_coefficients_reduce_to_sine_mode():
    """Fig. 1c with W0 = w1 and W1..W6 = w2 everywhere is Fig. 1b."""
    n = (8, 9, 7)
    R = 1
    nx, ny, nz = n
    k = (2, 3, 1)
    phi = np.zeros(wl.padded_shape(n, R))
    ix = np.sin(np.pi * k[0] * np.arange(1, nx + 1) / (nx + 1))
    iy = np.sin(np.pi * k[1] * np.arange(1, ny + 1) / (ny + 1))
    iz = np.sin(np.pi * k[2] * np.arange(1, nz + 1) / (nz + 1))
    phi[1:-1, 1:-1, 1:-1] = iz[:, None, None] * iy[None, :, None] * ix[None, None, :]
    W = np.empty((7,) + phi.shape)
    W[0] = 0.3
    W[1:] = 0.11
    mu = 0.3 + 2 * 0.11 * sum(np.cos(np.pi * k[i] / (n[i] + 1)) for i in range(3))
    T = 6
    _, u, _ = oracle.forward(J7_VAR, phi, phi, None, W, T)
    assert np.max(np.abs(u - mu ** T * phi)) <= 1e-14


# ---------------------------------------------------------------- P3 wave modes
def toeplitz_1d(N, diag, off):
    A = np.zeros((N, N))
    for i in range(N):
        A[i, i] = diag
        for r in range(1, 5):
            if i + r < N:
                A[i, i + r] = A[i + r, i] = off[r - 1]
    return A


def wave_mode_setup(n, modes, diag, off):
    """3D mode psi_i (x) psi_j (y) psi_k (z) of the separable operator
    T_x + T_y + T_z built from 1D truncated Toeplitz matrices (zero halo)."""
    nx, ny, nz = n
    ex, vx = np.linalg.eigh(toeplitz_1d(nx, diag, off))
    ey, vy = np.linalg.eigh(toeplitz_1d(ny, diag, off))
    ez, vz = np.linalg.eigh(toeplitz_1d(nz, diag, off))
    i, j, k = modes
    lam = ex[i] + ey[j] + ez[k]
    R = 4
    phi = np.zeros(wl.padded_shape(n, R))
    phi[R:-R, R:-R, R:-R] = vz[:, k][:, None, None] * vy[:, j][None, :, None] * vx[:, i][None, None, :]
    phi /= np.abs(phi).max()
    return phi, lam


def leapfrog_closed_form(alpha_lam, nsteps):
    """u^{n+1} = (2 + a) u^n - u^{n-1}, u^{-1} = u^0 = 1, with 2 cos(theta) = 2 + a:
    u^n = cos((n + 1/2) theta) / cos(theta / 2)."""
    theta = np.arccos(1.0 + alpha_lam / 2.0)
    return np.cos((nsteps + 0.5) * theta) / np.cos(theta / 2.0)


@pytest.mark.parametrize("modes", [(0, 0, 0), (3, 1, 5), (9, 8, 2)])
def test_w25_const_leapfrog_eigenmode(modes):
    n = (10, 9, 11)
    L8 = wl.L8_1D
    phi, lam = wave_mode_setup(n, modes, L8[0], L8[1:])
    w = wl.w25_const_weights(0.1)
    T = 40
    p, u, _ = oracle.forward(W25_CONST, phi, phi, w, None, T)
    assert np.max(np.abs(u - leapfrog_closed_form(0.1 * lam, T) * phi)) <= 1e-12
    assert np.max(np.abs(p - leapfrog_closed_form(0.1 * lam, T - 1) * phi)) <= 1e-12


def test_w25_var_and_alpha_with_constant_coefficients_reduce_to_closed_form():
    """Fig. 1d coefficients / Fig. 1e alpha array held constant in space give
    the same leapfrog closed form as the scalar-alpha stencil."""
    n = (9, 10, 8)
    L8 = wl.L8_1D
    phi, lam = wave_mode_setup(n, (2, 4, 1), L8[0], L8[1:])
    alpha = 0.09
    shape = phi.shape
    W = np.zeros((13,) + shape)
    W[0] = alpha * 3 * L8[0]
    for r in range(1, 5):
        for a in range(3):
            W[3 * (r - 1) + a + 1] = alpha * L8[r]
    T = 25
    ref = leapfrog_closed_form(alpha * lam, T) * phi
    _, u, _ = oracle.forward(W25_VAR, phi, phi, None, W, T)
    assert np.max(np.abs(u - ref)) <= 1e-12
    A = np.full((1,) + shape, alpha)
    _, u, _ = oracle.forward(W25_ALPHA, phi, phi, wl.w25_const_weights(1.0)[1:], A, T)
    assert np.max(np.abs(u - ref)) <= 1e-12


def test_j25_var_constant_coefficients_eigenmode():
    """Fig. 1d with spatially constant W is diagonal on the Toeplitz modes:
    u^T = (W0 + sum_a lam_a)^T phi with off-diagonals W_r, zero diagonal."""
    n = (9, 8, 10)
    off = [0.05, 0.03, 0.02, 0.01]
    phi, lam = wave_mode_setup(n, (1, 2, 3), 0.0, off)
    W = np.zeros((13,) + phi.shape)
    W[0] = 0.2
    for r in range(1, 5):
        for a in range(3):
            W[3 * (r - 1) + a + 1] = off[r - 1]
    T = 7
    _, u, _ = oracle.forward(J25_VAR, phi, phi, None, W, T)
    assert np.max(np.abs(u - (0.2 + lam) ** T * phi)) <= 1e-13


# ---------------------------------------------------------------- P4 impulses
@pytest.mark.parametrize("kind", ALL_KINDS)
def test_impulse_response_matches_offset_table(kind):
    """A unit impulse at interior point p gives, after one step,
    u'(p - o_k) = A_k(p - o_k) for every term k of Fig. 1 (plus 2 at p for
    wave kinds) and zero elsewhere."""
    rng = np.random.default_rng(7)
    R = oracle.RADIUS[kind]
    n = (13, 12, 14)
    shape = wl.padded_shape(n, R)
    p = (6, 5, 7)  # (x, y, z) interior, zero-based; p +- R stays interior
    u = np.zeros(shape)
    u[p[2] + R, p[1] + R, p[0] + R] = 1.0
    w = default_weights(kind)
    W = None
    expected = np.zeros(shape)
    if kind in (J7_VAR, W25_VAR, J25_VAR):
        W = rand_coeffs(kind, n, rng)
        table = OFFSETS_J7_VAR if kind == J7_VAR else offsets_25()
        for k, (dx, dy, dz) in table:
            q = (p[2] - dz + R, p[1] - dy + R, p[0] - dx + R)
            expected[q] += W[(k,) + q]
    elif kind == J7_CONST:
        for k, (dx, dy, dz) in OFFSETS_J7_VAR:
            q = (p[2] - dz + R, p[1] - dy + R, p[0] - dx + R)
            expected[q] += w[0] if k == 0 else w[1]
    else:  # W25_CONST, W25_ALPHA: alpha(q) * w_r at distance r
        if kind == W25_ALPHA:
            W = rand_coeffs(kind, n, rng)
            alpha_at = lambda q: W[(0,) + q]  # noqa: E731
            wts = w
        else:
            alpha_at = lambda q: w[0]  # noqa: E731
            wts = w[1:]
        for k, (dx, dy, dz) in offsets_25():
            q = (p[2] - dz + R, p[1] - dy + R, p[0] - dx + R)
            r = max(abs(dx), abs(dy), abs(dz))
            expected[q] += alpha_at(q) * wts[r]
    if oracle.SECOND_ORDER[kind]:
        expected[p[2] + R, p[1] + R, p[0] + R] += 2.0
    _, out, _ = oracle.forward(kind, np.zeros(shape), u, w, W, 1)
    assert np.count_nonzero(out) == np.count_nonzero(expected)
    np.testing.assert_allclose(out, expected, rtol=0, atol=4 * EPS)


def test_wave_kinds_subtract_previous_level():
    """u^{t-1} enters with coefficient -1 at the same point (Fig. 1e)."""
    R = 4
    n = (10, 10, 10)
    shape = wl.padded_shape(n, R)
    prev = np.zeros(shape)
    prev[R + 4, R + 5, R + 3] = 1.0
    for kind, w, W in [(W25_CONST, wl.w25_const_weights(0.1), None),
                       (W25_VAR, None, np.ones((13,) + shape)),
                       (W25_ALPHA, wl.w25_const_weights(0.1)[1:], np.ones((1,) + shape))]:
        _, out, _ = oracle.forward(kind, prev, np.zeros(shape), w, W, 1)
        expect = -prev
        np.testing.assert_array_equal(out, expect)


def laurent_power(wc, wf, T):
    """Exact coefficients of (wc + wf * sum_a (x_a + 1/x_a))^T as {(i,j,k): Fraction}."""
    poly = {(0, 0, 0): Fraction(1)}
    step = {(0, 0, 0): wc}
    for a in range(3):
        for s in (-1, 1):
            e = [0, 0, 0]
            e[a] = s
            step[tuple(e)] = wf
    for _ in range(T):
        new = {}
        for (i, j, k), c in poly.items():
            for (di, dj, dk), d in step.items():
                key = (i + di, j + dj, k + dk)
                new[key] = new.get(key, 0) + c * d
        poly = new
    return poly


def test_j7_multistep_impulse_is_laurent_power():
    """T steps of Fig. 1b from an impulse give the coefficients of the
    T-th power of its symbol, computed in exact rational arithmetic."""
    T = 4
    n = (11, 11, 11)
    R = 1
    u = np.zeros(wl.padded_shape(n, R))
    c = 5
    u[c + R, c + R, c + R] = 1.0
    _, out, _ = oracle.forward(J7_CONST, u, u, [0.4, 0.1], None, T)
    poly = laurent_power(Fraction(2, 5), Fraction(1, 10), T)
    expected = np.zeros_like(u)
    for (i, j, k), v in poly.items():
        expected[c + k + R, c + j + R, c + i + R] = float(v)
    np.testing.assert_allclose(out, expected, rtol=0, atol=1e-16)


# ---------------------------------------------------------------- P6 symmetry
@pytest.mark.parametrize("kind", [J7_CONST, W25_CONST])
@pytest.mark.parametrize("perm", [(1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)])
def test_axis_permutation_symmetry(kind, perm):
    """Isotropic constant-coefficient stencils commute with axis permutations."""
    rng = np.random.default_rng(11)
    R = oracle.RADIUS[kind]
    n = (12, 12, 12)
    u = rand_interior(n, R, rng)
    up = rand_interior(n, R, rng)
    w = default_weights(kind)
    p1, q1, _ = oracle.forward(kind, up, u, w, None, 3)
    p2, q2, _ = oracle.forward(kind, np.ascontiguousarray(up.transpose(perm)),
                               np.ascontiguousarray(u.transpose(perm)), w, None, 3)
    np.testing.assert_allclose(q2, q1.transpose(perm), rtol=0, atol=1e-13)
    np.testing.assert_allclose(p2, p1.transpose(perm), rtol=0, atol=1e-13)


# ---------------------------------------------------------------- P7 energy
def test_w25_const_discrete_energy_conserved():
    """For the leapfrog scheme with a symmetric operator A,
    E^{n+1/2} = |u^{n+1} - u^n|^2 - <u^{n+1}, A u^n> is constant; A u^n is
    read off the scheme itself as u^{n+1} - 2u^n + u^{n-1}."""
    rng = np.random.default_rng(5)
    R = 4
    n = (14, 13, 12)
    u0 = rand_interior(n, R, rng)
    um = rand_interior(n, R, rng) * 0.5 + u0 * 0.5
    w = wl.w25_const_weights(0.1)
    states = [um, u0]
    p, c = um, u0
    for _ in range(30):
        p, c, _ = oracle.forward(W25_CONST, p, c, w, None, 1)
        states.append(c)
    E = []
    for m in range(1, len(states) - 1):
        un1, un, unm = states[m + 1], states[m], states[m - 1]
        Au = un1 - 2 * un + unm
        E.append(np.sum((un1 - un) ** 2) - np.sum(un1 * Au))
    E = np.array(E)
    assert np.max(np.abs(E - E[0])) <= 1e-11 * max(1.0, abs(E[0]))


def test_w25_stability_bound():
    """alpha * max|symbol| <= 4 for the benchmark weights: no blow-up."""
    L8 = wl.L8_1D
    sym = 3 * (abs(L8[0]) + 2 * sum(abs(x) for x in L8[1:]))
    assert 0.1 * sym <= 4.0 and 0.12 * 1.1 * sym <= 4.0
    rng = np.random.default_rng(3)
    R = 4
    n = (12, 12, 12)
    u = rand_interior(n, R, rng)
    _, out, _ = oracle.forward(W25_CONST, u, u, wl.w25_const_weights(0.1), None, 200)
    assert np.abs(out).max() < 50.0


# ---------------------------------------------------------------- P8 adjoint
@pytest.mark.parametrize("kind", ALL_KINDS)
@pytest.mark.parametrize("T", [1, 4])
def test_adjoint_dot_product(kind, T):
    """<F_T(a, b), (x, y)> = <(a, b), F_T^T (x, y)> where F_T advances the
    state pair T steps and F_T^T runs the adjoint recursion.  For wave kinds
    the pair map M = [[0, I], [-I, 2I + A]] satisfies M^T = D N D with
    D = diag(-I, I) and N the adjoint pair step, so F_T^T (x, y) =
    (-l2, l1) for (l2, l1) = adjoint(-x, y)."""
    rng = np.random.default_rng(100 + kind + 10 * T)
    R = oracle.RADIUS[kind]
    n = (10, 9, 11)
    a, b, x, y = (rand_interior(n, R, rng) for _ in range(4))
    w = default_weights(kind)
    W = rand_coeffs(kind, n, rng, 0.01, 0.2) if oracle.NUM_ARRAYS[kind] else None
    pT, cT, _ = oracle.forward(kind, a, b, w, W, T)
    if oracle.SECOND_ORDER[kind]:
        l2, l1 = oracle.adjoint(kind, -x, y, w, W, T)
        lhs = np.sum(pT * x) + np.sum(cT * y)
        rhs = np.sum(a * -l2) + np.sum(b * l1)
    else:
        l2, l1 = oracle.adjoint(kind, x, y, w, W, T)
        lhs = np.sum(cT * y)
        rhs = np.sum(b * l1)
        if T >= 1:
            assert abs(np.sum(pT * y) - np.sum(b * l2)) <= 1e-13 * np.sum(np.abs(pT * y))
    assert abs(lhs - rhs) <= 1e-13 * max(1.0, np.sum(np.abs(pT * x)) + np.sum(np.abs(cT * y)))


def _fd_check(kind, n, T, rcv_z, seed, directions=2, w=None):
    rng = np.random.default_rng(seed)
    R = oracle.RADIUS[kind]
    u0 = rand_interior(n, R, rng)
    k = oracle.NUM_ARRAYS[kind]
    if kind == W25_VAR:
        v = rng.uniform(0.05, 0.12, size=(n[2], n[1], n[0]))
        W = wl.w25_var_coeffs(n, v, seed)
    else:
        W = rand_coeffs(kind, n, rng, 0.01, 0.14)
    d = rng.uniform(-0.1, 0.1, size=(T, n[1], n[0]))
    loss, du0, dW = oracle.loss_and_gradient(kind, u0, W, d, T, rcv_z, w=w)

    def L(u0_, W_):
        _, _, tr = oracle.forward(kind, u0_, u0_, w, W_, T, rcv_z=rcv_z)
        return oracle.receiver_loss(tr, d)[0]

    assert abs(L(u0, W) - loss) <= 1e-12 * abs(loss)
    for _ in range(directions):
        du = rand_interior(n, R, rng)
        h = 1e-4
        fd = (L(u0 + h * du, W) - L(u0 - h * du, W)) / (2 * h)
        an = np.sum(du0 * du)
        assert abs(fd - an) <= 1e-7 * max(abs(an), 1e-30) + 1e-14, (fd, an)
        for kk in range(k):
            dw = np.zeros_like(W)
            dw[kk] = rand_interior(n, R, rng) * np.abs(W[kk]).max()
            h = 1e-5
            fd = (L(u0, W + h * dw) - L(u0, W - h * dw)) / (2 * h)
            an = np.sum(dW * dw)
            assert abs(fd - an) <= 1e-6 * max(abs(an), abs(fd)) + 1e-14, (kk, fd, an)


@pytest.mark.parametrize("kind", VAR_KINDS)
def test_gradient_finite_differences_small(kind):
    w = default_weights(kind)
    _fd_check(kind, (10, 11, 12), 6, 3, seed=kind, directions=1, w=w)


def test_fwi_48_gradient_finite_differences():
    """The 48^3 copy of the differentiable wave workload: the gradient of the
    receiver misfit w.r.t. u0 and all 13 arrays matches central differences."""
    fw = wl.fwi(48, T=60, K=10, seed=0)
    _, _, d = oracle.forward(W25_VAR, fw.u0, fw.u0, None, fw.W_true, fw.T, rcv_z=fw.rcv_z, threads=4)
    loss, du0, dW = oracle.loss_and_gradient(W25_VAR, fw.u0, fw.W, d, fw.T, fw.rcv_z, threads=4)
    assert loss > 0
    rng = np.random.default_rng(9)
    R = 4

    def L(u0_, W_):
        _, _, tr = oracle.forward(W25_VAR, u0_, u0_, None, W_, fw.T, rcv_z=fw.rcv_z, threads=4)
        return oracle.receiver_loss(tr, d)[0]

    du = rand_interior(fw.n, R, rng)
    h = 1e-3
    fd = (L(fw.u0 + h * du, fw.W) - L(fw.u0 - h * du, fw.W)) / (2 * h)
    an = np.sum(du0 * du)
    assert abs(fd - an) <= 1e-6 * abs(an)
    for kk in (0, 1, 5, 12):
        dw = np.zeros_like(fw.W)
        dw[kk] = rand_interior(fw.n, R, rng) * np.abs(fw.W[kk]).max()
        h = 1e-6  # central-difference error is O(h^2): 6e-6 relative at 1e-5
        fd = (L(fw.u0, fw.W + h * dw) - L(fw.u0, fw.W - h * dw)) / (2 * h)
        an = np.sum(dW * dw)
        assert abs(fd - an) <= 1e-6 * max(abs(an), abs(fd)), (kk, fd, an)


def test_receiver_trace_is_plane_of_each_state():
    """trace[t] is u^{t+1} on the receiver plane (interior index rcv_z)."""
    w = wl.j7_const(8, 3)
    p, c = w.u_prev, w.u
    _, _, tr = oracle.forward(J7_CONST, p, c, w.w, None, 3, rcv_z=5)
    for t in range(3):
        p, c, _ = oracle.forward(J7_CONST, p, c, w.w, None, 1)
        np.testing.assert_array_equal(tr[t], c[5 + 1, 1:-1, 1:-1])


def test_threads_do_not_change_bits():
    w = wl.make(W25_VAR, 20, 3)
    a = oracle.forward(W25_VAR, w.u_prev, w.u, None, w.W, 3, threads=1)[1]
    b = oracle.forward(W25_VAR, w.u_prev, w.u, None, w.W, 3, threads=4)[1]
    np.testing.assert_array_equal(a, b)


def test_zero_steps_and_bad_arguments():
    w = wl.j7_const(6, 0)
    p, c, _ = oracle.forward(J7_CONST, w.u_prev, w.u, w.w, None, 0)
    np.testing.assert_array_equal(c, w.u)
    with pytest.raises(ValueError):
        oracle.forward(J7_CONST, w.u_prev, w.u, w.w, None, -1)


def test_halo_never_written():
    rng = np.random.default_rng(2)
    for kind in ALL_KINDS:
        R = oracle.RADIUS[kind]
        n = (9, 9, 9)
        u = rand_interior(n, R, rng)
        W = rand_coeffs(kind, n, rng) if oracle.NUM_ARRAYS[kind] else None
        p, c, _ = oracle.forward(kind, u, u, default_weights(kind), W, 3)
        mask = np.ones(c.shape, bool)
        mask[R:-R, R:-R, R:-R] = False
        assert not c[mask].any() and not p[mask].any()
