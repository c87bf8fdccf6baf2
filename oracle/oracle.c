/*
 * oracle.c -- plain FP64 CPU definition of the stencil sweeps.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the CUDA
 * library: only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no code, header or constant with the CUDA
 * path.  Every loop is the naive update order of the paper (Sect. 3.1 and
 * Fig. 1): one full sweep over the interior per time step, t outermost, then
 * z, y, x with x fastest.  No blocking, no fusion, no reordering.  Compiled
 * with -O2 -ffp-contract=off so that no multiply-add is contracted and the
 * result is the same on x86_64 and aarch64.  The optional OpenMP pragma only
 * splits the (z, y) loops of one sweep across threads; every lattice update is
 * still computed independently by the same expression, so the result does not
 * depend on the thread count.
 *
 * Lattice and storage (Sect. 3.1): Omega[t][z][y][x], x unit stride.  The
 * interior is 1..N in every axis (Fig. 1 loop bounds), surrounded by a halo of
 * width R that holds zero Dirichlet values and is never written.  Arrays are
 * halo padded: extents (nz+2R, ny+2R, nx+2R).  Coefficient arrays W[k] use the
 * same padded layout; their halo values are never read.
 *
 * Kinds (numbers are part of the interface):
 *   1  7-point constant coefficients, first order in time      (Fig. 1b)
 *      w = {w1, w2}:  u' = w1*u + w2*(x pair) + w2*(y pair) + w2*(z pair)
 *   2  7-point variable coefficients, first order in time      (Fig. 1c)
 *      W[0..6] at the updated point: centre, x-1, x+1, y-1, y+1, z-1, z+1
 *   3  25-point constant coefficients, second order in time    (Fig. 1e, scalar alpha)
 *      w = {alpha, w0, w1, w2, w3, w4};  w0 is the 3D centre weight
 *      u^{t+1} = 2u^t - u^{t-1} + alpha*[w0*u^t + sum_r w_r*(pairs along x, y, z)]
 *   4  25-point variable coefficients, second order in time
 *      (Fig. 1d coefficient structure with the time scheme of Fig. 1e)
 *      u^{t+1} = 2u^t - u^{t-1} + W0*u^t + sum_{r,a} W[3(r-1)+a+1]*(pair at distance r on axis a)
 *   5  25-point variable coefficients, first order in time     (Fig. 1d)
 *      u' = W0*u + sum_{r,a} W[3(r-1)+a+1]*(pair at distance r on axis a)
 *   6  25-point, second order in time, domain-sized alpha      (Fig. 1e)
 *      w = {w0, w1, w2, w3, w4}, W[0] = alpha array
 *   axis a: 0 = x, 1 = y, 2 = z.
 *
 * Time-state convention (both directions): the call receives the pair
 * (prev, cur) and returns the pair advanced by T steps.  Forward: on entry
 * (u_prev, u) = (u^{-1}, u^0) -- u_prev is ignored by first-order kinds -- and
 * on return (u_prev, u) = (u^{T-1}, u^T).  T = 0 leaves both untouched.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OK_ 0
#define EINVAL_ -1
#define ENOMEM_ -3

enum { J7_CONST = 1, J7_VAR = 2, W25_CONST = 3, W25_VAR = 4, J25_VAR = 5, W25_ALPHA = 6 };

static int kind_radius(int kind) {
    switch (kind) {
    case J7_CONST: case J7_VAR: return 1;
    case W25_CONST: case W25_VAR: case J25_VAR: case W25_ALPHA: return 4;
    default: return -1;
    }
}

static int second_order(int kind) {
    return kind == W25_CONST || kind == W25_VAR || kind == W25_ALPHA;
}

int oracle_num_arrays(int kind) {
    switch (kind) {
    case J7_VAR: return 7;
    case W25_VAR: case J25_VAR: return 13;
    case W25_ALPHA: return 1;
    default: return 0;
    }
}

int oracle_num_weights(int kind) {
    switch (kind) {
    case J7_CONST: return 2;
    case W25_CONST: return 6;
    case W25_ALPHA: return 5;
    default: return 0;
    }
}

typedef struct {
    int64_t nx, ny, nz;
    int R;
    int64_t px, py, pz;    /* padded extents */
    int64_t sx, sy, sz;    /* strides in elements */
    int64_t n;             /* padded element count */
} geom_t;

static geom_t make_geom(int64_t nx, int64_t ny, int64_t nz, int R) {
    geom_t g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.R = R;
    g.px = nx + 2 * R; g.py = ny + 2 * R; g.pz = nz + 2 * R;
    g.sx = 1; g.sy = g.px; g.sz = g.px * g.py;
    g.n = g.px * g.py * g.pz;
    return g;
}

static int check_args(int kind, int64_t nx, int64_t ny, int64_t nz, int R, int64_t T) {
    if (kind_radius(kind) < 0 || R != kind_radius(kind)) return EINVAL_;
    if (nx < 1 || ny < 1 || nz < 1 || T < 0) return EINVAL_;
    return OK_;
}

/* Stride of axis a (0 = x, 1 = y, 2 = z). */
static int64_t axis_stride(const geom_t *g, int a) {
    return a == 0 ? g->sx : (a == 1 ? g->sy : g->sz);
}

/* One forward lattice update at padded linear index i (Fig. 1). */
static double update_point(int kind, const geom_t *g, const double *c, const double *p,
                           const double *w, const double *W, int64_t i) {
    const int64_t sx = g->sx, sy = g->sy, sz = g->sz, n = g->n;
    switch (kind) {
    case J7_CONST:
        return w[0] * c[i]
             + w[1] * (c[i - sx] + c[i + sx])
             + w[1] * (c[i - sy] + c[i + sy])
             + w[1] * (c[i - sz] + c[i + sz]);
    case J7_VAR:
        return W[0 * n + i] * c[i]
             + W[1 * n + i] * c[i - sx]
             + W[2 * n + i] * c[i + sx]
             + W[3 * n + i] * c[i - sy]
             + W[4 * n + i] * c[i + sy]
             + W[5 * n + i] * c[i - sz]
             + W[6 * n + i] * c[i + sz];
    case W25_CONST: {
        double s = w[1] * c[i];
        for (int r = 1; r <= 4; ++r)
            s += w[1 + r] * ((c[i - r * sx] + c[i + r * sx])
                           + (c[i - r * sy] + c[i + r * sy])
                           + (c[i - r * sz] + c[i + r * sz]));
        return 2.0 * c[i] - p[i] + w[0] * s;
    }
    case W25_ALPHA: {
        double s = w[0] * c[i];
        for (int r = 1; r <= 4; ++r)
            s += w[r] * ((c[i - r * sx] + c[i + r * sx])
                       + (c[i - r * sy] + c[i + r * sy])
                       + (c[i - r * sz] + c[i + r * sz]));
        return 2.0 * c[i] - p[i] + W[i] * s;
    }
    case W25_VAR:
    case J25_VAR: {
        double s = W[i] * c[i];
        for (int r = 1; r <= 4; ++r)
            for (int a = 0; a < 3; ++a) {
                const int64_t st = r * axis_stride(g, a);
                s += W[(int64_t)(3 * (r - 1) + a + 1) * n + i] * (c[i - st] + c[i + st]);
            }
        if (kind == W25_VAR) return 2.0 * c[i] - p[i] + s;
        return s;
    }
    }
    return 0.0;
}

static double *dup_array(const double *src, int64_t n) {
    double *d = (double *)malloc((size_t)n * sizeof(double));
    if (d) memcpy(d, src, (size_t)n * sizeof(double));
    return d;
}

int oracle_forward(int kind, int64_t nx, int64_t ny, int64_t nz, int R,
                   double *u_prev, double *u, const double *w, const double *W,
                   int64_t T, double *trace, int64_t rcv_z, int nthreads) {
    int st = check_args(kind, nx, ny, nz, R, T);
    if (st) return st;
    if (trace && (rcv_z < 0 || rcv_z >= nz)) return EINVAL_;
    if (T == 0) return OK_;
    const geom_t g = make_geom(nx, ny, nz, R);
    double *prev = dup_array(u_prev, g.n), *cur = dup_array(u, g.n), *next = dup_array(u_prev, g.n);
    if (!prev || !cur || !next) { free(prev); free(cur); free(next); return ENOMEM_; }
    (void)nthreads;
    for (int64_t t = 0; t < T; ++t) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads) if (nthreads > 1)
        for (int64_t z = R; z < R + nz; ++z)
            for (int64_t y = R; y < R + ny; ++y)
                for (int64_t x = R; x < R + nx; ++x) {
                    const int64_t i = z * g.sz + y * g.sy + x;
                    next[i] = update_point(kind, &g, cur, prev, w, W, i);
                }
        if (trace) {
            double *plane = trace + t * nx * ny;
            const int64_t z = rcv_z + R;
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x)
                    plane[y * nx + x] = next[z * g.sz + (y + R) * g.sy + (x + R)];
        }
        double *tmp = prev; prev = cur; cur = next; next = tmp;
    }
    memcpy(u_prev, prev, (size_t)g.n * sizeof(double));
    memcpy(u, cur, (size_t)g.n * sizeof(double));
    free(prev); free(cur); free(next);
    return OK_;
}

/* ---------------------------------------------------------------------------
 * Adjoint.  The forward update of every kind is a linear map
 *     u'(p) = sum_k A_k(p) * u(p + o_k)      (+ 2u(p) - u_prev(p) for wave kinds)
 * over interior points p.  Its transpose gathers from the source points:
 *     (A^T y)(q) = sum_k A_k(q - o_k) * y(q - o_k),
 * where only interior source points q - o_k contribute.
 *
 * Loss L = sum_n l_n(u^n) with explicit partials g^n = dL/du^n; the receiver
 * misfit has g^n = P^T r^n, r^n the residual on the receiver plane.
 *   first-order kinds:   lam^n = g^n + A^T lam^{n+1}
 *   second-order kinds:  lam^n = g^n + 2 lam^{n+1} + A^T lam^{n+1} - lam^{n+2}
 * Coefficient gradients, summed over the steps n of the call:
 *   dL/dA_k(x) += lam^{n+1}(x) * (d(A u^n)(x) / dA_k(x)).
 *
 * Call convention mirrors the forward one.  On entry (lam_next, lam) =
 * (lam^{m+1}, lam^m) with g^m already included in lam^m; the call runs steps
 * n = m-1 down to m-T and returns (lam_next, lam) = (lam^{m-T+1}, lam^{m-T}).
 * states[i] = u^{m-T+i} (contiguous, T padded fields), residual[i] = r^{m-T+i}
 * on the receiver plane (T interior planes, may be NULL), grad (may be NULL)
 * holds the coefficient gradients in the coefficient layout and is
 * accumulated into (interior entries only).
 * ------------------------------------------------------------------------- */

static int interior(const geom_t *g, int64_t z, int64_t y, int64_t x) {
    return z >= g->R && z < g->R + g->nz && y >= g->R && y < g->R + g->ny &&
           x >= g->R && x < g->R + g->nx;
}

/* (A^T y)(q) for the spatial operator A (without the 2u - u_prev part). */
static double adjoint_point(int kind, const geom_t *g, const double *y, const double *w,
                            const double *W, int64_t z, int64_t yy, int64_t x) {
    const int64_t n = g->n;
    const int64_t q = z * g->sz + yy * g->sy + x;
    double s = 0.0;
    switch (kind) {
    case J7_CONST: {
        /* symmetric: A^T = A (centre w1, six faces w2); halo y is zero */
        s = w[0] * y[q];
        for (int a = 0; a < 3; ++a) {
            const int64_t st = axis_stride(g, a);
            for (int sgn = -1; sgn <= 1; sgn += 2) {
                const int64_t dz = (a == 2) ? sgn : 0, dy = (a == 1) ? sgn : 0, dx = (a == 0) ? sgn : 0;
                if (interior(g, z + dz, yy + dy, x + dx)) s += w[1] * y[q + sgn * st];
            }
        }
        return s;
    }
    case J7_VAR: {
        /* forward offsets o_k: 0, -x, +x, -y, +y, -z, +z.  Source point of
           term k is q - o_k. */
        static const int off[7][3] = {{0,0,0},{-1,0,0},{1,0,0},{0,-1,0},{0,1,0},{0,0,-1},{0,0,1}};
        for (int k = 0; k < 7; ++k) {
            const int64_t sxo = -off[k][0], syo = -off[k][1], szo = -off[k][2];
            if (!interior(g, z + szo, yy + syo, x + sxo)) continue;
            const int64_t src = q + szo * g->sz + syo * g->sy + sxo * g->sx;
            s += W[(int64_t)k * n + src] * y[src];
        }
        return s;
    }
    case W25_CONST:
    case W25_ALPHA: {
        /* A = diag(alpha) * L with L symmetric, so A^T y = L (alpha * y). */
        const double wc = (kind == W25_CONST) ? w[1] : w[0];
        const double *wr = (kind == W25_CONST) ? w + 1 : w;  /* wr[r], r = 1..4 */
        const double al = (kind == W25_CONST) ? w[0] : 0.0;
#define AY(idx) ((kind == W25_CONST) ? al * y[idx] : W[idx] * y[idx])
        s = wc * AY(q);
        for (int r = 1; r <= 4; ++r)
            for (int a = 0; a < 3; ++a) {
                const int64_t st = r * axis_stride(g, a);
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int64_t d = sgn * r;
                    const int64_t dz = (a == 2) ? d : 0, dy = (a == 1) ? d : 0, dx = (a == 0) ? d : 0;
                    if (interior(g, z + dz, yy + dy, x + dx)) s += wr[r] * AY(q + sgn * st);
                }
            }
#undef AY
        return s;
    }
    case W25_VAR:
    case J25_VAR: {
        s = W[q] * y[q];
        for (int r = 1; r <= 4; ++r)
            for (int a = 0; a < 3; ++a) {
                const int64_t k = 3 * (r - 1) + a + 1;
                const int64_t st = r * axis_stride(g, a);
                for (int sgn = -1; sgn <= 1; sgn += 2) {
                    const int64_t d = sgn * r;
                    const int64_t dz = (a == 2) ? d : 0, dy = (a == 1) ? d : 0, dx = (a == 0) ? d : 0;
                    if (interior(g, z + dz, yy + dy, x + dx)) {
                        const int64_t src = q + sgn * st;
                        s += W[k * n + src] * y[src];
                    }
                }
            }
        return s;
    }
    }
    return 0.0;
}

/* Gradient contribution of one step at interior index i:
   grad_k(i) += lam1(i) * d(A u)(i)/dA_k(i). */
static void grad_point(int kind, const geom_t *g, const double *u, const double *lam1,
                       const double *w, double *grad, int64_t i) {
    const int64_t n = g->n;
    const double l = lam1[i];
    switch (kind) {
    case J7_VAR: {
        const int64_t o[7] = {0, -g->sx, g->sx, -g->sy, g->sy, -g->sz, g->sz};
        for (int k = 0; k < 7; ++k) grad[(int64_t)k * n + i] += l * u[i + o[k]];
        return;
    }
    case W25_VAR:
    case J25_VAR: {
        grad[i] += l * u[i];
        for (int r = 1; r <= 4; ++r)
            for (int a = 0; a < 3; ++a) {
                const int64_t st = r * axis_stride(g, a);
                grad[(int64_t)(3 * (r - 1) + a + 1) * n + i] += l * (u[i - st] + u[i + st]);
            }
        return;
    }
    case W25_ALPHA: {
        double s = w[0] * u[i];
        for (int r = 1; r <= 4; ++r)
            s += w[r] * ((u[i - r * g->sx] + u[i + r * g->sx])
                       + (u[i - r * g->sy] + u[i + r * g->sy])
                       + (u[i - r * g->sz] + u[i + r * g->sz]));
        grad[i] += l * s;
        return;
    }
    default:
        return;
    }
}

int oracle_adjoint(int kind, int64_t nx, int64_t ny, int64_t nz, int R,
                   double *lam_next, double *lam, const double *w, const double *W,
                   int64_t T, const double *states, const double *residual, int64_t rcv_z,
                   double *grad, int nthreads) {
    int st = check_args(kind, nx, ny, nz, R, T);
    if (st) return st;
    if (residual && (rcv_z < 0 || rcv_z >= nz)) return EINVAL_;
    if (grad && oracle_num_arrays(kind) == 0) return EINVAL_;
    if (T == 0) return OK_;
    if (!states && grad) return EINVAL_;
    const geom_t g = make_geom(nx, ny, nz, R);
    const int so = second_order(kind);
    /* l2 = lam^{n+2}, l1 = lam^{n+1}, l0 = lam^n (being built) */
    double *l2 = dup_array(lam_next, g.n), *l1 = dup_array(lam, g.n), *l0 = dup_array(lam_next, g.n);
    if (!l2 || !l1 || !l0) { free(l2); free(l1); free(l0); return ENOMEM_; }
    (void)nthreads;
    for (int64_t j = 1; j <= T; ++j) {
        const int64_t idx = T - j;  /* step n = m - j uses states[idx] = u^n */
        if (grad) {
            const double *un = states + idx * g.n;
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads) if (nthreads > 1)
            for (int64_t z = R; z < R + nz; ++z)
                for (int64_t y = R; y < R + ny; ++y)
                    for (int64_t x = R; x < R + nx; ++x)
                        grad_point(kind, &g, un, l1, w, grad, z * g.sz + y * g.sy + x);
        }
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads) if (nthreads > 1)
        for (int64_t z = R; z < R + nz; ++z)
            for (int64_t y = R; y < R + ny; ++y)
                for (int64_t x = R; x < R + nx; ++x) {
                    const int64_t i = z * g.sz + y * g.sy + x;
                    double v = adjoint_point(kind, &g, l1, w, W, z, y, x);
                    if (so) v = 2.0 * l1[i] + v - l2[i];
                    l0[i] = v;
                }
        if (residual) {
            const double *plane = residual + idx * nx * ny;
            const int64_t z = rcv_z + R;
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x)
                    l0[z * g.sz + (y + R) * g.sy + (x + R)] += plane[y * nx + x];
        }
        double *tmp = l2; l2 = l1; l1 = l0; l0 = tmp;
    }
    memcpy(lam_next, l2, (size_t)g.n * sizeof(double));
    memcpy(lam, l1, (size_t)g.n * sizeof(double));
    free(l2); free(l1); free(l0);
    return OK_;
}
