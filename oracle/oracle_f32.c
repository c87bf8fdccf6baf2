/*
 * oracle_f32.c -- the forward sweep of oracle.c evaluated in FP32.
 *
 * TEST INFRASTRUCTURE ONLY (same rules as oracle.c: loaded by the tests, the
 * smoke check and the CPU-baseline leg of the benchmark; shares no code with
 * the CUDA path).
 *
 * The FP32 mode of the method stores fields and coefficients in FP32 and
 * accumulates in FP32.  This file is the plain definition of that mode: the
 * naive sweep of Fig. 1 (Sect. 3.1), t outermost, then z, y, x, every
 * update the same expression in the same order of terms as oracle.c, with
 * float storage and float arithmetic (-ffp-contract=off: every product and
 * sum rounded to float separately, no multiply-add contraction).  Its
 * difference from the FP64 oracle on the same (FP32-rounded) inputs is the
 * rounding error of an FP32 evaluation, the scale against which the tests
 * measure the error of the GPU's FP32 sweeps.
 *
 * Kinds, layout and the time-state convention are those of oracle.c.  The
 * weights w are given in FP64 and rounded to float once.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { K_J7_CONST = 1, K_J7_VAR = 2, K_W25_CONST = 3, K_W25_VAR = 4, K_J25_VAR = 5, K_W25_ALPHA = 6 };

static int radius_f32(int kind) {
    if (kind == K_J7_CONST || kind == K_J7_VAR) return 1;
    if (kind >= K_W25_CONST && kind <= K_W25_ALPHA) return 4;
    return -1;
}

typedef struct {
    int64_t nx, ny, nz, px, py, pz, sy, sz, n;
    int R;
} grid32_t;

/* One update at padded index i; lam = the FP32 weights. */
static float point_f32(int kind, const grid32_t *g, const float *u, const float *up, const float *lam,
                       const float *A, int64_t i) {
    const int64_t ax[3] = {1, g->sy, g->sz};
    const int64_t n = g->n;
    switch (kind) {
    case K_J7_CONST:
        return lam[0] * u[i]
             + lam[1] * (u[i - 1] + u[i + 1])
             + lam[1] * (u[i - g->sy] + u[i + g->sy])
             + lam[1] * (u[i - g->sz] + u[i + g->sz]);
    case K_J7_VAR:
        return A[i] * u[i]
             + A[n + i] * u[i - 1]
             + A[2 * n + i] * u[i + 1]
             + A[3 * n + i] * u[i - g->sy]
             + A[4 * n + i] * u[i + g->sy]
             + A[5 * n + i] * u[i - g->sz]
             + A[6 * n + i] * u[i + g->sz];
    case K_W25_CONST:
    case K_W25_ALPHA: {
        /* W25_CONST: lam = {alpha, w0..w4}; W25_ALPHA: lam = {w0..w4}, alpha = A */
        const float *wt = kind == K_W25_CONST ? lam + 1 : lam;
        float acc = wt[0] * u[i];
        for (int r = 1; r <= 4; ++r)
            acc += wt[r] * ((u[i - r] + u[i + r])
                          + (u[i - r * g->sy] + u[i + r * g->sy])
                          + (u[i - r * g->sz] + u[i + r * g->sz]));
        const float al = kind == K_W25_CONST ? lam[0] : A[i];
        return 2.0f * u[i] - up[i] + al * acc;
    }
    case K_W25_VAR:
    case K_J25_VAR: {
        float acc = A[i] * u[i];
        for (int r = 1; r <= 4; ++r)
            for (int a = 0; a < 3; ++a) {
                const int64_t d = r * ax[a];
                acc += A[(int64_t)(3 * (r - 1) + a + 1) * n + i] * (u[i - d] + u[i + d]);
            }
        return kind == K_W25_VAR ? 2.0f * u[i] - up[i] + acc : acc;
    }
    }
    return 0.0f;
}

/* Same arguments and conventions as oracle_forward, in FP32. */
int oracle_forward_f32(int kind, int64_t nx, int64_t ny, int64_t nz, int R, float *u_prev, float *u,
                       const double *w, int nw, const float *W, int64_t T, float *trace, int64_t rcv_z,
                       int nthreads) {
    if (radius_f32(kind) < 0 || R != radius_f32(kind) || nx < 1 || ny < 1 || nz < 1 || T < 0) return -1;
    if (trace && (rcv_z < 0 || rcv_z >= nz)) return -1;
    if (nw < 0 || nw > 8) return -1;
    if (T == 0) return 0;
    grid32_t g;
    g.nx = nx; g.ny = ny; g.nz = nz; g.R = R;
    g.px = nx + 2 * R; g.py = ny + 2 * R; g.pz = nz + 2 * R;
    g.sy = g.px; g.sz = g.px * g.py; g.n = g.sz * g.pz;
    float lam[8] = {0};
    for (int k = 0; k < nw; ++k) lam[k] = (float)w[k];
    const size_t bytes = (size_t)g.n * sizeof(float);
    float *prev = (float *)malloc(bytes), *cur = (float *)malloc(bytes), *next = (float *)malloc(bytes);
    if (!prev || !cur || !next) { free(prev); free(cur); free(next); return -3; }
    memcpy(prev, u_prev, bytes);
    memcpy(cur, u, bytes);
    memcpy(next, u_prev, bytes);
    (void)nthreads;
    for (int64_t t = 0; t < T; ++t) {
#pragma omp parallel for collapse(2) schedule(static) num_threads(nthreads) if (nthreads > 1)
        for (int64_t z = R; z < R + nz; ++z)
            for (int64_t y = R; y < R + ny; ++y)
                for (int64_t x = R; x < R + nx; ++x) {
                    const int64_t i = z * g.sz + y * g.sy + x;
                    next[i] = point_f32(kind, &g, cur, prev, lam, W, i);
                }
        if (trace) {
            float *plane = trace + t * nx * ny;
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x)
                    plane[y * nx + x] = next[(rcv_z + R) * g.sz + (y + R) * g.sy + (x + R)];
        }
        float *tmp = prev; prev = cur; cur = next; next = tmp;
    }
    memcpy(u_prev, prev, bytes);
    memcpy(u, cur, bytes);
    free(prev); free(cur); free(next);
    return 0;
}
