// plain_impl.cuh -- the plain one-step-per-sweep kernels (forward and adjoint);
// instantiated per dtype by plain_f32.cu and plain_f64.cu.
//
// One launch applies one time level to the whole lattice: the naive update
// order of the paper (Sect. 4.1, "naive" approach, Fig. 4a) with the spatial
// blocking of Sect. 3.3 mapped to a GPU 2.5D scheme:
//
//  * a CTA owns a TX x TY tile of (x, y) columns and marches along z through
//    a chunk of planes;
//  * every input plane of the stencil field (tile plus a halo of R in x and
//    y) is staged in shared memory with cp.async, PD planes ahead of use, in
//    a ring of NS = R + 2 + PD plane slots (one __syncthreads per plane);
//  * each thread owns one x column and NR consecutive y rows; the 2R + 1
//    planes it needs along z live in a register ring (the loop is unrolled
//    by 2R + 1 so ring slots are compile-time registers), y neighbours inside
//    the thread's own rows come from that ring, the rest and the x
//    neighbours from the shared-memory plane;
//  * the second-order kinds update in place (u^{t+1} overwrites u^{t-1}, as
//    the paper's two-copy storage does, Sect. 3.1); first-order kinds write a
//    separate array.
//
// The adjoint launch is the same kernel with the transposed operator:
// (A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k) reads each coefficient at the
// source point of its term (a shifted, coalesced load); the constant kinds
// are symmetric and reuse the forward update.
#pragma once
#include "common.cuh"
#include "plain.cuh"

namespace stc {

template <typename T, int KIND, bool ADJ, int TX, int BY, int NR, int PD>
__global__ void __launch_bounds__(TX * BY)
plain_sweep_kernel(const SweepArgs<T> a) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int TY = BY * NR;
    constexpr int SW = TX + 2 * R;       // shared plane row length
    constexpr int SH = TY + 2 * R;       // shared plane rows
    constexpr int SPLANE = SW * SH;
    constexpr int NS = R + 2 + PD;       // shared plane slots
    constexpr int RING = 2 * R + 1;      // register ring depth along z
    constexpr int NT = TX * BY;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);

    const Geom g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * TX + tx;
    const int x0 = blockIdx.x * TX;            // interior x of the tile = padded x of its halo start
    const int y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int x = x0 + tx;                      // interior x of this thread
    const bool xok = x < g.nx;

    const int qs = z0 - R, qe = z1 + R;         // interior indices of the planes read

    auto issue = [&](int q) {
        const T *src = a.u + (int64_t)(q + R) * g.sz;
        T *dst = sm + cmod(q - qs, NS) * SPLANE;
#pragma unroll 4
        for (int e = tid; e < SPLANE; e += NT) {
            const int r = e / SW, c = e - r * SW;
            const int gy = y0 + r, gx = x0 + c;  // padded coordinates
            if (gy < g.py && gx < g.px) cp_async<sizeof(T)>(dst + e, src + (int64_t)gy * g.sy + gx);
        }
    };

    T ring[RING][NR];
#pragma unroll
    for (int i = 0; i < RING; ++i)
#pragma unroll
        for (int jr = 0; jr < NR; ++jr) ring[i][jr] = T(0);

#pragma unroll
    for (int i = 0; i < PD; ++i) {
        if (qs + i < qe) issue(qs + i);
        cp_async_commit();
    }

    const T s0 = T(a.s.c[0]), s1 = T(a.s.c[1]), s2 = T(a.s.c[2]);
    const T s3 = T(a.s.c[3]), s4 = T(a.s.c[4]), s5 = T(a.s.c[5]);
    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4; (void)s5;

    for (int qb = qs; qb < qe; qb += RING) {
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            const int q = qb + j;
            if (q < qe) {
                if (q + PD < qe) issue(q + PD);
                cp_async_commit();
                cp_async_wait<PD>();
                __syncthreads();

                const T *sq = sm + cmod(q - qs, NS) * SPLANE;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) ring[j][jr] = sq[(ty * NR + jr + R) * SW + tx + R];

                const int z = q - R;
                if (z >= z0) {
                    const T *sp = sm + cmod(z - qs, NS) * SPLANE;
                    constexpr int jc = cmod(j - R, RING);   // ring slot of plane z
                    const int64_t zrow = (int64_t)(z + R) * g.sz;
#pragma unroll
                    for (int jr = 0; jr < NR; ++jr) {
                        const int y = y0 + ty * NR + jr;
                        if (!xok || y >= g.ny) continue;
                        const int lr = ty * NR + jr + R;    // shared row of this point
                        const int64_t idx = zrow + (int64_t)(y + R) * g.sy + (x + R);
                        const T c = ring[jc][jr];
                        // neighbours: [r-1][0] = minus side, [r-1][1] = plus side
                        T xn[R][2], yn[R][2], zn[R][2];
#pragma unroll
                        for (int r = 1; r <= R; ++r) {
                            xn[r - 1][0] = sp[lr * SW + tx + R - r];
                            xn[r - 1][1] = sp[lr * SW + tx + R + r];
                            if (jr - r >= 0) yn[r - 1][0] = ring[jc][jr - r];
                            else yn[r - 1][0] = sp[(lr - r) * SW + tx + R];
                            if (jr + r < NR) yn[r - 1][1] = ring[jc][jr + r];
                            else yn[r - 1][1] = sp[(lr + r) * SW + tx + R];
                            zn[r - 1][0] = ring[cmod(j - R - r, RING)][jr];
                            zn[r - 1][1] = ring[cmod(j - R + r, RING)][jr];
                        }
                        T v;
                        if constexpr (KIND == J7_CONST) {
                            // s0 = w1, s1 = w2 (Fig. 1b); symmetric, so also the adjoint
                            v = s0 * c + s1 * (((xn[0][0] + xn[0][1]) + (yn[0][0] + yn[0][1])) + (zn[0][0] + zn[0][1]));
                        } else if constexpr (KIND == J7_VAR) {
                            const T *Wp = a.W + idx;
                            const int64_t n = g.nfield, sy = g.sy, sz = g.sz;
                            (void)sy; (void)sz;
                            if constexpr (!ADJ) {
                                // Fig. 1c: W0 c + W1 x- + W2 x+ + W3 y- + W4 y+ + W5 z- + W6 z+
                                v = Wp[0] * c;
                                v = fma(Wp[1 * n], xn[0][0], v);
                                v = fma(Wp[2 * n], xn[0][1], v);
                                v = fma(Wp[3 * n], yn[0][0], v);
                                v = fma(Wp[4 * n], yn[0][1], v);
                                v = fma(Wp[5 * n], zn[0][0], v);
                                v = fma(Wp[6 * n], zn[0][1], v);
                            } else {
                                // transpose: term k is gathered from q - o_k
                                v = Wp[0] * c;
                                v = fma(Wp[1 * n + 1], xn[0][1], v);
                                v = fma(Wp[2 * n - 1], xn[0][0], v);
                                v = fma(Wp[3 * n + sy], yn[0][1], v);
                                v = fma(Wp[4 * n - sy], yn[0][0], v);
                                v = fma(Wp[5 * n + sz], zn[0][1], v);
                                v = fma(Wp[6 * n - sz], zn[0][0], v);
                            }
                        } else if constexpr (KIND == W25_CONST) {
                            // folded Fig. 1e: s0 = 2 + alpha w0, s1..s4 = alpha w_r
                            T acc = s0 * c - a.u_prev[idx];
                            const T wr[4] = {s1, s2, s3, s4};
#pragma unroll
                            for (int r = 0; r < 4; ++r)
                                acc = fma(wr[r], ((xn[r][0] + xn[r][1]) + (yn[r][0] + yn[r][1])) + (zn[r][0] + zn[r][1]), acc);
                            v = acc;
                        } else if constexpr (KIND == W25_ALPHA) {
                            // Fig. 1e: 2u - u_prev + alpha(x) [w0 u + sum_r w_r S_r]
                            const T wr[4] = {s1, s2, s3, s4};
                            if constexpr (!ADJ) {
                                T s = s0 * c;
#pragma unroll
                                for (int r = 0; r < 4; ++r)
                                    s = fma(wr[r], ((xn[r][0] + xn[r][1]) + (yn[r][0] + yn[r][1])) + (zn[r][0] + zn[r][1]), s);
                                v = fma(a.W[idx], s, T(2) * c - a.u_prev[idx]);
                            } else {
                                // A^T y = L (alpha y): alpha read at every source point
                                const T *Ap = a.W + idx;
                                const int64_t sy = g.sy, sz = g.sz;
                                T s = s0 * (Ap[0] * c);
#pragma unroll
                                for (int r = 0; r < 4; ++r) {
                                    const int d = r + 1;
                                    T pr = Ap[-d] * xn[r][0];
                                    pr = fma(Ap[d], xn[r][1], pr);
                                    pr = fma(Ap[-d * sy], yn[r][0], pr);
                                    pr = fma(Ap[d * sy], yn[r][1], pr);
                                    pr = fma(Ap[-d * sz], zn[r][0], pr);
                                    pr = fma(Ap[d * sz], zn[r][1], pr);
                                    s = fma(wr[r], pr, s);
                                }
                                v = s + (T(2) * c - a.u_prev[idx]);
                            }
                        } else {  // W25_VAR, J25_VAR (Fig. 1d coefficient structure)
                            const T *Wp = a.W + idx;
                            const int64_t n = g.nfield, sy = g.sy, sz = g.sz;
                            (void)sy; (void)sz;
                            T acc = Wp[0] * c;
                            if constexpr (WAVE) acc = fma(T(2), c, acc) - a.u_prev[idx];
#pragma unroll
                            for (int r = 0; r < 4; ++r) {
                                const int d = r + 1;
                                (void)d;
                                const T *Wx = Wp + (3 * r + 1) * n;
                                const T *Wy = Wp + (3 * r + 2) * n;
                                const T *Wz = Wp + (3 * r + 3) * n;
                                if constexpr (!ADJ) {
                                    acc = fma(Wx[0], xn[r][0] + xn[r][1], acc);
                                    acc = fma(Wy[0], yn[r][0] + yn[r][1], acc);
                                    acc = fma(Wz[0], zn[r][0] + zn[r][1], acc);
                                } else {
                                    acc = fma(Wx[-d], xn[r][0], acc);
                                    acc = fma(Wx[d], xn[r][1], acc);
                                    acc = fma(Wy[-d * sy], yn[r][0], acc);
                                    acc = fma(Wy[d * sy], yn[r][1], acc);
                                    acc = fma(Wz[-d * sz], zn[r][0], acc);
                                    acc = fma(Wz[d * sz], zn[r][1], acc);
                                }
                            }
                            v = acc;
                        }
                        if (z == a.rcv_z) {
                            const int64_t pidx = (int64_t)y * g.nx + x;
                            if (a.inject) v += a.inject[pidx];
                            if (a.trace) a.trace[pidx] = v;
                        }
                        if (dbg_store_ok(a.dbg, g, idx)) a.out[idx] = v;
                    }
                }
            }
        });
    }
}

// ---------------------------------------------------------------- streaming forward
// One forward level (also the adjoint of the symmetric constant kinds).
// The kernel is written for few instructions per lattice update:
//  * the field plane q + PD (tile plus halo) is staged by cp.async in
//    iteration q into a ring of NSU = M (2R+1) >= R + 2 + PD plane slots
//    (a plane is read until R iterations after it arrives and must not be
//    overwritten while a slower thread still reads it).  Each thread copies
//    fixed rows (ty + i BY) of its column (and of one halo column when
//    tx < 2R): in-plane offsets and bounds masks are computed once, a
//    plane costs one 64-bit base per iteration;
//  * slot numbers are compile-time constants within a block of 2R+1
//    iterations (the z loop is unrolled by 2R+1, which also makes the z
//    register ring static), plus the block's parity when M > 1;
//  * the per-point inputs of an output plane (u^{t-1}, coefficients, no
//    halo) are loaded into registers one iteration before use;
//  * receiver trace / residual injection are handled once per plane.
// ADJ: the adjoint sweep of a variable-coefficient kind.  The transpose
// gathers each term's coefficient at its source point,
// (A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k); those NC coefficient values per
// point (7 for Fig. 1c, 25 for the 25-point kinds) are the per-point inputs
// that travel one iteration ahead in registers.
template <int KIND, bool ADJ> struct PointCoeffs { static constexpr int value = KindTraits<KIND>::NARR; };
template <int KIND> struct PointCoeffs<KIND, true> {
    static constexpr int value = KindTraits<KIND>::NARR == 0 ? 0 : (KindTraits<KIND>::R == 1 ? 7 : 25);
};

template <typename T, int KIND, int TX, int BY, int NR, int PD, bool STAGE = false, bool ADJ = false>
__global__ void __launch_bounds__(TX * BY)
plain_stream_kernel(const SweepArgs<T> a) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int NA = PointCoeffs<KIND, ADJ>::value;
    static_assert(!(ADJ && STAGE), "the adjoint sweep keeps its per-point inputs in registers");
    constexpr int TY = BY * NR;
    constexpr int SW = TX + 2 * R;
    constexpr int SH = TY + 2 * R;
    constexpr int SPLANE = SW * SH;
    constexpr int RING = 2 * R + 1;
    constexpr int M = (R + 2 + PD + RING - 1) / RING;
    constexpr int NSU = M * RING;
    constexpr int NLR = (SH + BY - 1) / BY;       // rows each thread copies
    constexpr int NPO = (WAVE ? 1 : 0) + NA;
    constexpr int NPB = NPO > 0 ? NPO : 1;
    static_assert(2 * R <= TX, "halo columns are copied by the first 2R threads");
    static_assert(NLR <= 32 && NR <= 32, "bit masks");

    // STAGE: per-point inputs also travel through the cp.async pipeline, in
    // a ring of NSO = PD + 2 output-plane slots ([NPO][TY][TX] each)
    constexpr int OT = TX * TY;
    constexpr int NSO = PD + 2;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *su = reinterpret_cast<T *>(smem_raw);       // [NSU][SH][SW]
    T *so = su + NSU * SPLANE;                     // STAGE: [NSO][NPO][TY][TX]
    (void)so;

    const Geom g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int x0 = blockIdx.x * TX;
    const int y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int x = x0 + tx;
    const int qs = z0 - R, qe = z1 + R;
    const int sy = (int)g.sy;

    // ---- copy plan of this thread (padded coordinates, in-plane offsets)
    const int goff0 = (y0 + ty) * sy + x0 + tx;
    uint32_t mmain = 0, mhalo = 0;
#pragma unroll
    for (int i = 0; i < NLR; ++i) {
        const int r = ty + i * BY, gy = y0 + r;
        if (r < SH && gy < g.py) {
            if (x0 + tx < g.px) mmain |= 1u << i;
            if (tx < 2 * R && x0 + TX + tx < g.px) mhalo |= 1u << i;
        }
    }
    auto issue = [&](int q, T *dst) {
        const T *pb = a.u + (int64_t)(q + R) * g.sz + goff0;
        T *d = dst + ty * SW + tx;
#pragma unroll
        for (int i = 0; i < NLR; ++i) {
            if (mmain & (1u << i)) cp_async<sizeof(T)>(d + i * BY * SW, pb + i * BY * sy);
            if (mhalo & (1u << i)) cp_async<sizeof(T)>(d + i * BY * SW + TX, pb + i * BY * sy + TX);
        }
    };

    // ---- this thread's output rows
    const int pofs0 = (y0 + ty * NR + R) * sy + x + R;     // in-plane offset of row 0
    uint32_t rowok = 0;
#pragma unroll
    for (int jr = 0; jr < NR; ++jr)
        if (x < g.nx && y0 + ty * NR + jr < g.ny) rowok |= 1u << jr;

    T pin[NPB][NR], pnx[NPB][NR];
    auto load_point_inputs = [&](int z) {
        if constexpr (NPO > 0) {
            if (z >= z1) return;
            const int64_t base = (int64_t)(z + R) * g.sz + pofs0;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (!(rowok & (1u << jr))) continue;
                const int64_t off = base + jr * sy;
                if constexpr (WAVE) pnx[0][jr] = a.u_prev[off];
                constexpr int CO = WAVE ? 1 : 0;
                if constexpr (!ADJ) {
#pragma unroll
                    for (int t = 0; t < NA; ++t) pnx[CO + t][jr] = a.W[off + t * g.nfield];
                } else if constexpr (R == 1) {
                    // source points of Fig. 1c's terms: q, q+x, q-x, q+y, q-y, q+z, q-z
                    const int64_t n = g.nfield, sz = g.sz;
                    pnx[CO + 0][jr] = a.W[off];
                    pnx[CO + 1][jr] = a.W[off + n + 1];
                    pnx[CO + 2][jr] = a.W[off + 2 * n - 1];
                    pnx[CO + 3][jr] = a.W[off + 3 * n + sy];
                    pnx[CO + 4][jr] = a.W[off + 4 * n - sy];
                    pnx[CO + 5][jr] = a.W[off + 5 * n + sz];
                    pnx[CO + 6][jr] = a.W[off + 6 * n - sz];
                } else {
                    // 25-point kinds: centre, then per (r, axis) the coefficient at
                    // q - r e_a and at q + r e_a (alpha for the alpha-array kind)
                    const int64_t n = g.nfield;
                    const int64_t st3[3] = {1, (int64_t)sy, g.sz};
                    pnx[CO][jr] = a.W[off];
#pragma unroll
                    for (int r = 1; r <= 4; ++r)
#pragma unroll
                        for (int ax = 0; ax < 3; ++ax) {
                            const int64_t arr = (KIND == W25_ALPHA) ? 0 : (int64_t)(3 * (r - 1) + ax + 1) * n;
                            const int64_t d = r * st3[ax];
                            pnx[CO + 1 + 2 * (3 * (r - 1) + ax)][jr] = a.W[off + arr - d];
                            pnx[CO + 2 + 2 * (3 * (r - 1) + ax)][jr] = a.W[off + arr + d];
                        }
                }
            }
        }
    };

    // STAGE: copies of the per-point inputs of output plane z into slot `o`
    auto issue_points = [&](int z, int o) {
        if constexpr (STAGE && NPO > 0) {
            if (z < z0 || z >= z1) return;
            const int64_t base = (int64_t)(z + R) * g.sz + pofs0;
            T *d = so + o * (NPO * OT) + (ty * NR) * TX + tx;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (!(rowok & (1u << jr))) continue;
                const int64_t off = base + jr * sy;
                if constexpr (WAVE) cp_async<sizeof(T)>(d + jr * TX, a.u_prev + off);
#pragma unroll
                for (int t = 0; t < NA; ++t)
                    cp_async<sizeof(T)>(d + ((WAVE ? 1 : 0) + t) * OT + jr * TX, a.W + off + t * g.nfield);
            }
        }
    };

    T ring[RING][NR];
#pragma unroll
    for (int i = 0; i < RING; ++i)
#pragma unroll
        for (int jr = 0; jr < NR; ++jr) ring[i][jr] = T(0);
#pragma unroll
    for (int t = 0; t < NPB; ++t)
#pragma unroll
        for (int jr = 0; jr < NR; ++jr) { pin[t][jr] = T(0); pnx[t][jr] = T(0); }

    // prologue: planes qs .. qs+PD-1 into slots 0 .. PD-1 (and, staged, the
    // per-point inputs of their output planes)
#pragma unroll
    for (int i = 0; i < PD; ++i) {
        if (qs + i < qe) {
            issue(qs + i, su + i * SPLANE);
            issue_points(qs + i - R, i % NSO);
        }
        cp_async_commit();
    }
    if constexpr (!STAGE) load_point_inputs(z0);

    const T s0 = T(a.s.c[0]), s1 = T(a.s.c[1]), s2 = T(a.s.c[2]);
    const T s3 = T(a.s.c[3]), s4 = T(a.s.c[4]);
    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4;

    int blk = 0;   // (qb - qs) / RING modulo M
    for (int qb = qs; qb < qe; qb += RING) {
        T *const slots = su + blk * RING * SPLANE;          // slot of the block's first plane
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            const int q = qb + j;
            if (q >= qe) return;
            const int z = q - R;
            if constexpr (NPO > 0 && !STAGE) {
                if (z >= z0) {
#pragma unroll
                    for (int t = 0; t < NPO; ++t)
#pragma unroll
                        for (int jr = 0; jr < NR; ++jr) pin[t][jr] = pnx[t][jr];
                    load_point_inputs(z + 1);
                }
            }
            // slot of plane q + PD
            {
                T *dst = slots + (j + PD) * SPLANE;
                if (j + PD >= NSU - blk * RING) dst -= NSU * SPLANE;
                if (q + PD < qe) {
                    issue(q + PD, dst);
                    issue_points(q + PD - R, (q + PD - qs) % NSO);
                }
            }
            cp_async_commit();
            cp_async_wait<PD>();
            __syncthreads();
            if constexpr (STAGE && NPO > 0) {
                if (z >= z0) {
                    const T *sop = so + ((q - qs) % NSO) * (NPO * OT) + (ty * NR) * TX + tx;
#pragma unroll
                    for (int t = 0; t < NPO; ++t)
#pragma unroll
                        for (int jr = 0; jr < NR; ++jr) pin[t][jr] = sop[t * OT + jr * TX];
                }
            }

            const T *sq = slots + j * SPLANE;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) ring[j][jr] = sq[(ty * NR + jr + R) * SW + tx + R];
            if (z < z0) return;

            const T *sp = slots + (j - R) * SPLANE;               // plane z = q - R
            if (j - R < -blk * RING) sp += NSU * SPLANE;
            constexpr int jc = cmod(j - R, RING);
            T *outp = a.out + (int64_t)(z + R) * g.sz + pofs0;
            const T *rowp = sp + (ty * NR + R) * SW + tx + R;   // this thread's first row, centre column
            T res[NR];
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                const T *cp = rowp + jr * SW;
                const T c = ring[jc][jr];
                T xn[R][2], yn[R][2], zn[R][2];
#pragma unroll
                for (int d = 1; d <= R; ++d) {
                    xn[d - 1][0] = cp[-d];
                    xn[d - 1][1] = cp[d];
                    if (jr - d >= 0) yn[d - 1][0] = ring[jc][jr - d];
                    else yn[d - 1][0] = cp[-d * SW];
                    if (jr + d < NR) yn[d - 1][1] = ring[jc][jr + d];
                    else yn[d - 1][1] = cp[d * SW];
                    zn[d - 1][0] = ring[cmod(j - R - d, RING)][jr];
                    zn[d - 1][1] = ring[cmod(j - R + d, RING)][jr];
                }
                constexpr int CO = WAVE ? 1 : 0;   // per-point input index of the first coefficient
                (void)CO;
                const T pv = WAVE ? pin[0][jr] : T(0);
                (void)pv;
                T v;
                if constexpr (ADJ && KIND == J7_VAR) {
                    v = pin[CO + 0][jr] * c;
                    v = fma(pin[CO + 1][jr], xn[0][1], v);
                    v = fma(pin[CO + 2][jr], xn[0][0], v);
                    v = fma(pin[CO + 3][jr], yn[0][1], v);
                    v = fma(pin[CO + 4][jr], yn[0][0], v);
                    v = fma(pin[CO + 5][jr], zn[0][1], v);
                    v = fma(pin[CO + 6][jr], zn[0][0], v);
                } else if constexpr (ADJ && KIND == W25_ALPHA) {
                    const T wr[4] = {s1, s2, s3, s4};
                    T sacc = s0 * (pin[CO][jr] * c);
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int b = CO + 1 + 6 * d;
                        T pr = pin[b][jr] * xn[d][0];
                        pr = fma(pin[b + 1][jr], xn[d][1], pr);
                        pr = fma(pin[b + 2][jr], yn[d][0], pr);
                        pr = fma(pin[b + 3][jr], yn[d][1], pr);
                        pr = fma(pin[b + 4][jr], zn[d][0], pr);
                        pr = fma(pin[b + 5][jr], zn[d][1], pr);
                        sacc = fma(wr[d], pr, sacc);
                    }
                    v = sacc + (T(2) * c - pv);
                } else if constexpr (ADJ) {  // W25_VAR, J25_VAR
                    T acc = pin[CO][jr] * c;
                    if constexpr (WAVE) acc = fma(T(2), c, acc) - pv;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        const int b = CO + 1 + 6 * d;
                        acc = fma(pin[b][jr], xn[d][0], acc);
                        acc = fma(pin[b + 1][jr], xn[d][1], acc);
                        acc = fma(pin[b + 2][jr], yn[d][0], acc);
                        acc = fma(pin[b + 3][jr], yn[d][1], acc);
                        acc = fma(pin[b + 4][jr], zn[d][0], acc);
                        acc = fma(pin[b + 5][jr], zn[d][1], acc);
                    }
                    v = acc;
                } else if constexpr (KIND == J7_CONST) {
                    v = s0 * c + s1 * (((xn[0][0] + xn[0][1]) + (yn[0][0] + yn[0][1])) + (zn[0][0] + zn[0][1]));
                } else if constexpr (KIND == J7_VAR) {
                    v = pin[0][jr] * c;
                    v = fma(pin[1][jr], xn[0][0], v);
                    v = fma(pin[2][jr], xn[0][1], v);
                    v = fma(pin[3][jr], yn[0][0], v);
                    v = fma(pin[4][jr], yn[0][1], v);
                    v = fma(pin[5][jr], zn[0][0], v);
                    v = fma(pin[6][jr], zn[0][1], v);
                } else if constexpr (KIND == W25_CONST) {
                    T acc = s0 * c - pv;
                    const T wr[4] = {s1, s2, s3, s4};
#pragma unroll
                    for (int d = 0; d < 4; ++d)
                        acc = fma(wr[d], ((xn[d][0] + xn[d][1]) + (yn[d][0] + yn[d][1])) + (zn[d][0] + zn[d][1]), acc);
                    v = acc;
                } else if constexpr (KIND == W25_ALPHA) {
                    const T wr[4] = {s1, s2, s3, s4};
                    T s = s0 * c;
#pragma unroll
                    for (int d = 0; d < 4; ++d)
                        s = fma(wr[d], ((xn[d][0] + xn[d][1]) + (yn[d][0] + yn[d][1])) + (zn[d][0] + zn[d][1]), s);
                    v = fma(pin[CO][jr], s, T(2) * c - pv);
                } else {  // W25_VAR, J25_VAR
                    T acc = pin[CO][jr] * c;
                    if constexpr (WAVE) acc = fma(T(2), c, acc) - pv;
#pragma unroll
                    for (int d = 0; d < 4; ++d) {
                        acc = fma(pin[CO + 3 * d + 1][jr], xn[d][0] + xn[d][1], acc);
                        acc = fma(pin[CO + 3 * d + 2][jr], yn[d][0] + yn[d][1], acc);
                        acc = fma(pin[CO + 3 * d + 3][jr], zn[d][0] + zn[d][1], acc);
                    }
                    v = acc;
                }
                res[jr] = v;
            }
            if (z == a.rcv_z) {
                const int64_t pl = (int64_t)(y0 + ty * NR) * g.nx + x;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    if (!(rowok & (1u << jr))) continue;
                    if (a.inject) res[jr] += a.inject[pl + jr * g.nx];
                    if (a.trace) a.trace[pl + jr * g.nx] = res[jr];
                }
            }
#pragma unroll
            for (int jr = 0; jr < NR; ++jr)
                if ((rowok & (1u << jr)) && dbg_store_ok(a.dbg, g, (outp - a.out) + (int64_t)jr * sy))
                    outp[jr * sy] = res[jr];
        });
        blk = (blk + 1 == M) ? 0 : blk + 1;
    }
}

template <typename T, int KIND, int TX, int BY, int NR, int PD, bool STAGE = false>
constexpr size_t stream_smem() {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int TY = BY * NR;
    constexpr int RING = 2 * R + 1;
    constexpr int M = (R + 2 + PD + RING - 1) / RING;
    constexpr int NPO = (KindTraits<KIND>::WAVE ? 1 : 0) + KindTraits<KIND>::NARR;
    return sizeof(T) * ((size_t)(M * RING) * (TX + 2 * R) * (TY + 2 * R) +
                        (STAGE ? (size_t)(PD + 2) * NPO * TX * TY : 0));
}

// Grid: tiles of TX x TY columns times z chunks, chunks sized for about four
// waves of CTAs and at least 8R planes (each chunk re-reads 2R planes).
template <typename K>
static cudaError_t launch_grid(K kern, size_t smem, int TX, int BY, int TY, int R, const SweepArgs<void> *,
                               int nx, int ny, int nz, int num_sms, int *zchunk, dim3 *grid) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TX * BY, smem);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int gx = (nx + TX - 1) / TX, gy = (ny + TY - 1) / TY;
    const int64_t want = (int64_t)num_sms * blocks_per_sm * 4;
    const int64_t tiles = (int64_t)gx * gy;
    int nzc = (int)((want + tiles - 1) / tiles);
    const int min_chunk = 8 * R;
    if (nzc < 1) nzc = 1;
    if ((nz + nzc - 1) / nzc < min_chunk) nzc = (nz + min_chunk - 1) / min_chunk;
    if (nzc < 1) nzc = 1;
    *zchunk = (nz + nzc - 1) / nzc;
    *grid = dim3(gx, gy, (nz + *zchunk - 1) / *zchunk);
    return cudaSuccess;
}

template <typename T, int KIND, bool ADJ, int TX, int BY, int NR, int PD>
static cudaError_t launch_cfg(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int TY = BY * NR;
    constexpr int NS = R + 2 + PD;
    constexpr size_t smem = sizeof(T) * (size_t)NS * (TX + 2 * R) * (TY + 2 * R);
    auto kern = plain_sweep_kernel<T, KIND, ADJ, TX, BY, NR, PD>;
    SweepArgs<T> b = a;
    dim3 grid;
    cudaError_t e = launch_grid(kern, smem, TX, BY, TY, R, nullptr, a.g.nx, a.g.ny, a.g.nz, num_sms, &b.zchunk, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, dim3(TX, BY, 1), smem, st>>>(b);
    return cudaGetLastError();
}

template <typename T, int KIND, int TX, int BY, int NR, int PD, bool STAGE = false, bool ADJ = false>
static cudaError_t launch_stream(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int TY = BY * NR;
    constexpr size_t smem = stream_smem<T, KIND, TX, BY, NR, PD, STAGE>();
    static_assert(smem <= 227 * 1024, "shared memory per CTA");
    auto kern = plain_stream_kernel<T, KIND, TX, BY, NR, PD, STAGE, ADJ>;
    SweepArgs<T> b = a;
    dim3 grid;
    cudaError_t e = launch_grid(kern, smem, TX, BY, TY, R, nullptr, a.g.nx, a.g.ny, a.g.nz, num_sms, &b.zchunk, &grid);
    if (e != cudaSuccess) return e;
    kern<<<grid, dim3(TX, BY, 1), smem, st>>>(b);
    return cudaGetLastError();
}

}  // namespace stc
