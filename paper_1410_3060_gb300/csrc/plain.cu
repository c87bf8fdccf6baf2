// plain.cu -- the plain one-step-per-sweep kernels (forward and adjoint).
//
// One launch applies one time level to the whole lattice: the naive update
// order of the paper (Sect. 4.1, "naive" approach, Fig. 4a) with the spatial
// blocking of Sect. 3 mapped to a GPU 2.5D scheme:
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
                        a.out[idx] = v;
                    }
                }
            }
        });
    }
}

// ---------------------------------------------------------------- launch
template <typename T, int KIND, bool ADJ, int TX, int BY, int NR, int PD>
static cudaError_t launch_cfg(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int TY = BY * NR;
    constexpr int NS = R + 2 + PD;
    constexpr size_t smem = sizeof(T) * (size_t)NS * (TX + 2 * R) * (TY + 2 * R);
    auto kern = plain_sweep_kernel<T, KIND, ADJ, TX, BY, NR, PD>;
    static bool configured = false;  // per instantiation
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    SweepArgs<T> b = a;
    const int gx = (a.g.nx + TX - 1) / TX, gy = (a.g.ny + TY - 1) / TY;
    // z chunks: enough CTAs for several waves, chunks of at least 4R planes
    int blocks_per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, TX * BY, smem);
    if (blocks_per_sm < 1) blocks_per_sm = 1;
    const int64_t want = (int64_t)num_sms * blocks_per_sm * 4;
    int64_t tiles = (int64_t)gx * gy;
    int nzc = (int)((want + tiles - 1) / tiles);
    const int min_chunk = 8 * R;
    nzc = nzc < 1 ? 1 : nzc;
    if ((a.g.nz + nzc - 1) / nzc < min_chunk) nzc = (a.g.nz + min_chunk - 1) / min_chunk;
    if (nzc < 1) nzc = 1;
    b.zchunk = (a.g.nz + nzc - 1) / nzc;
    const int gz = (a.g.nz + b.zchunk - 1) / b.zchunk;
    dim3 grid(gx, gy, gz), block(TX, BY, 1);
    kern<<<grid, block, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename T, int KIND, bool ADJ>
static cudaError_t launch_kind(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    constexpr int R = KindTraits<KIND>::R;
    if constexpr (sizeof(T) == 4) {
        if constexpr (R == 1) return launch_cfg<T, KIND, ADJ, 64, 4, 8, 2>(a, st, num_sms);
        else return launch_cfg<T, KIND, ADJ, 32, 8, 4, 2>(a, st, num_sms);
    } else {
        if constexpr (R == 1) return launch_cfg<T, KIND, ADJ, 32, 8, 4, 2>(a, st, num_sms);
        else return launch_cfg<T, KIND, ADJ, 32, 8, 2, 2>(a, st, num_sms);
    }
}

template <typename T>
cudaError_t launch_plain(int kind, bool adjoint, const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    switch (kind) {
    case J7_CONST: return launch_kind<T, J7_CONST, false>(a, st, num_sms);      // symmetric
    case W25_CONST: return launch_kind<T, W25_CONST, false>(a, st, num_sms);    // symmetric
    case J7_VAR: return adjoint ? launch_kind<T, J7_VAR, true>(a, st, num_sms) : launch_kind<T, J7_VAR, false>(a, st, num_sms);
    case W25_VAR: return adjoint ? launch_kind<T, W25_VAR, true>(a, st, num_sms) : launch_kind<T, W25_VAR, false>(a, st, num_sms);
    case J25_VAR: return adjoint ? launch_kind<T, J25_VAR, true>(a, st, num_sms) : launch_kind<T, J25_VAR, false>(a, st, num_sms);
    case W25_ALPHA: return adjoint ? launch_kind<T, W25_ALPHA, true>(a, st, num_sms) : launch_kind<T, W25_ALPHA, false>(a, st, num_sms);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_plain<float>(int, bool, const SweepArgs<float> &, cudaStream_t, int);
template cudaError_t launch_plain<double>(int, bool, const SweepArgs<double> &, cudaStream_t, int);

}  // namespace stc
