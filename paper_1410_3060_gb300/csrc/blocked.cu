// blocked.cu -- temporally blocked passes: B time levels per sweep over HBM.
//
// Wavefront temporal blocking (paper Sect. 4.1) combined with diamond tiling
// in y (Sect. 4.2 / 4.3, the CATS2 shape: diamond tiles in y, wavefront in
// z), re-designed for a GPU SM:
//
//  * Wavefront in z.  A CTA marches through a chunk of z planes.  At step q
//    it receives input plane q, and level k (k = 1..B) updates plane
//    q - kR: the frontline has slope -1/R (Sect. 4.1), so level k consumes
//    planes of level k-1 that were produced in this or earlier steps.
//    Each thread owns one x column and NR consecutive y rows; for every
//    level it keeps the 2R+1 planes of the previous level its column needs
//    in a register ring (the step loop is unrolled by 2R+1 so ring slots are
//    registers).  The x/y neighbours of level k's centre plane are exchanged
//    through one shared-memory plane per level (double buffered: one
//    __syncthreads per step).  The "thread group sharing a cache" of the
//    multi-thread wavefront (Sect. 4.4, MWD) is the CTA sharing its SM's
//    registers and shared memory; all its warps advance the frontline
//    together, synchronised once per plane.
//  * x is tiled with an overlapped halo of B*R columns (the paper leaves x
//    untiled; an SM cannot hold a full row times the wavefront).
//  * y, scheme OVL: overlapped tiles (halo B*R rows), one launch per pass.
//  * y, scheme DIAMOND: split (diamond) tiling, two launches per pass.
//    Phase A tiles [jW, (j+1)W) shrink by R rows per level on both sides;
//    they write the first and last 2R rows of every intermediate level to
//    band buffers.  Phase B tiles, centred on the A-tile boundaries jW,
//    grow by R rows per level on both sides, reading their outer 2R rows of
//    each level from the bands; an A tile of one pass and the B tile above
//    it form the diamond of Fig. 5 (slopes +-1/R, two parents), and B tiles
//    at the domain ends are the half diamonds.  No y row is computed twice.
//  * Levels are never stored except the last one (and the one before it,
//    which is the next pass's u^{t-1}), the receiver trace of every level,
//    and the diamond edge bands.  Points outside the interior hold the zero
//    Dirichlet value at every level.
//  * z is split into chunks for parallelism; each chunk recomputes a ramp
//    of (B-k)R planes of level k on each side (overlapped in z).
//
// The update of one point is the same expression as the plain kernel
// (plain.cu), so blocked and plain results agree to rounding.
#include "blocked.cuh"

namespace stc {

enum Phase { PH_OVL = 0, PH_A = 1, PH_B = 2 };

template <int PHASE, int B, int R, int RY>
struct Rows {
    // rows (region coordinates) level k computes
    __device__ static constexpr bool computed(int k, int ry) {
        return PHASE == PH_B ? (ry >= (B + 1 - k) * R && ry < (B + 1 + k) * R)
                             : (ry >= k * R && ry < RY - k * R);
    }
    // rows of level k this tile owns (stores / traces)
    __device__ static constexpr bool owned(int k, int ry) {
        return PHASE == PH_OVL ? (ry >= B * R && ry < RY - B * R) : computed(k, ry);
    }
    // phase A: rows of level k written to the band buffer (1 <= k < B)
    __device__ static constexpr bool band_store(int k, int ry) {
        return PHASE == PH_A && ((ry >= k * R && ry < (k + 2) * R) || (ry >= RY - (k + 2) * R && ry < RY - k * R));
    }
    // phase B: rows of level k read from the band buffer (1 <= k < B)
    __device__ static constexpr bool band_load(int k, int ry) {
        return PHASE == PH_B && ((ry >= (B - 1 - k) * R && ry < (B + 1 - k) * R) ||
                                 (ry >= (B + 1 + k) * R && ry < (B + 3 + k) * R));
    }
};

template <typename T, int KIND, int PHASE, int B, int TX, int BY, int NR>
__global__ void __launch_bounds__(TX * BY)
blocked_kernel(const BlockedArgs<T> a) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int RY = BY * NR;
    constexpr int RING = 2 * R + 1;
    constexpr int PX = TX + 2 * R;      // shared plane pitch (R pad on each side)
    constexpr int PY = RY + 2 * R;
    constexpr int PLANE = PX * PY;
    static_assert(PHASE != PH_B || RY == 2 * (B + 1) * R, "phase B region is 2(B+1)R rows");
    static_assert(PHASE == PH_B || RY >= 2 * B * R, "tile must hold the trapezoid");
    using Rw = Rows<PHASE, B, R, RY>;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sm = reinterpret_cast<T *>(smem_raw);  // [B][2][PLANE]

    const Geom g = a.g;
    const int tx = threadIdx.x, ty = threadIdx.y;
    constexpr int TXO = TX - 2 * B * R;
    const int X0 = (int)blockIdx.x * TXO - B * R;
    int Y0;
    if constexpr (PHASE == PH_OVL) Y0 = (int)blockIdx.y * (RY - 2 * B * R) - B * R;
    else if constexpr (PHASE == PH_A) Y0 = (int)blockIdx.y * RY;
    else Y0 = (int)blockIdx.y * a.wA - (B + 1) * R;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int x = X0 + tx;
    const bool xin = x >= 0 && x < g.nx;
    const bool xown = xin && tx >= B * R && tx < TX - B * R;
    const bool xmem = x >= -R && x < g.nx + R;   // inside the padded array

    const int qs = z0 - B * R, qe = z1 + B * R;
    const int64_t plane_elems = (int64_t)g.nx * g.ny;

    T ring[B][RING][NR];
#pragma unroll
    for (int k = 0; k < B; ++k)
#pragma unroll
        for (int i = 0; i < RING; ++i)
#pragma unroll
            for (int j = 0; j < NR; ++j) ring[k][i][j] = T(0);

    // level-0 input of the next step and (second order) u^{t-1} of level 1
    T pre[NR], preP[NR];
    auto load_level0 = [&](int q) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const int y = Y0 + ty * NR + j;
            const bool ok = xmem && y >= -R && y < g.ny + R && q >= -R && q < g.nz + R;
            pre[j] = ok ? a.u[(int64_t)(q + R) * g.sz + (int64_t)(y + R) * g.sy + (x + R)] : T(0);
        }
    };
    auto load_prev = [&](int z) {
#pragma unroll
        for (int j = 0; j < NR; ++j) {
            const int y = Y0 + ty * NR + j;
            const bool ok = xin && y >= 0 && y < g.ny && z >= 0 && z < g.nz;
            preP[j] = ok ? a.u_prev[(int64_t)(z + R) * g.sz + (int64_t)(y + R) * g.sy + (x + R)] : T(0);
        }
    };
    load_level0(qs);
    if constexpr (WAVE) load_prev(qs - R);

    const T s0 = T(a.s.c[0]), s1 = T(a.s.c[1]), s2 = T(a.s.c[2]);
    const T s3 = T(a.s.c[3]), s4 = T(a.s.c[4]);
    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4;

    int par = 0;
    for (int qb = qs; qb < qe; qb += RING) {
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            const int q = qb + j;
            if (q >= qe) return;
            // (a) level-0 front (plane q) into level 1's ring
            T curP[NR];
#pragma unroll
            for (int r = 0; r < NR; ++r) { ring[0][j][r] = pre[r]; curP[r] = preP[r]; }
            // (b) prefetch the next step's inputs
            if (q + 1 < qe) {
                load_level0(q + 1);
                if constexpr (WAVE) load_prev(q + 1 - R);
            }
            // (c) centre planes of every level into shared memory
            static_for<B>([&](auto kk) {
                constexpr int k = decltype(kk)::value + 1;
                if (q < qs + 2 * k * R) return;
                T *buf = sm + ((k - 1) * 2 + par) * PLANE;
                constexpr int jc = cmod(j - k * R, RING);
#pragma unroll
                for (int r = 0; r < NR; ++r) buf[(ty * NR + r + R) * PX + tx + R] = ring[k - 1][jc][r];
            });
            __syncthreads();
            // (d) levels 1..B
            static_for<B>([&](auto kk) {
                constexpr int k = decltype(kk)::value + 1;
                if (q < qs + 2 * k * R) return;
                const int z = q - k * R;
                const bool zin = z >= 0 && z < g.nz;
                const bool zown = z >= z0 && z < z1;
                const T *sp = sm + ((k - 1) * 2 + par) * PLANE;
                // ring slot of plane z (all rings index planes alike); ring[k-1]
                // holds level k-1 around z, level k's result enters ring[k] there
                constexpr int jc = cmod(j - k * R, RING);
                const int64_t zoff = (int64_t)(z + R) * g.sz;
#pragma unroll
                for (int r = 0; r < NR; ++r) {
                    const int ry = ty * NR + r;
                    const int y = Y0 + ry;
                    const bool in = xin && zin && y >= 0 && y < g.ny;
                    const int64_t idx = zoff + (int64_t)(y + R) * g.sy + (x + R);
                    T v = T(0);
                    if (Rw::computed(k, ry)) {
                        if (in) {
                            const int lr = ry + R;
                            const T c = ring[k - 1][jc][r];
                            T xn[R][2], yn[R][2], zn[R][2];
#pragma unroll
                            for (int d = 1; d <= R; ++d) {
                                xn[d - 1][0] = sp[lr * PX + tx + R - d];
                                xn[d - 1][1] = sp[lr * PX + tx + R + d];
                                if (r - d >= 0) yn[d - 1][0] = ring[k - 1][jc][r - d];
                                else yn[d - 1][0] = sp[(lr - d) * PX + tx + R];
                                if (r + d < NR) yn[d - 1][1] = ring[k - 1][jc][r + d];
                                else yn[d - 1][1] = sp[(lr + d) * PX + tx + R];
                                zn[d - 1][0] = ring[k - 1][cmod(j - k * R - d, RING)][r];
                                zn[d - 1][1] = ring[k - 1][cmod(j - k * R + d, RING)][r];
                            }
                            // u^{t-1} of this level: level k-2 at plane z
                            T pv = T(0);
                            if constexpr (WAVE) {
                                if constexpr (k == 1) pv = curP[r];
                                else pv = ring[k - 2][cmod(j - k * R, RING)][r];
                            }
                            (void)pv;
                            if constexpr (KIND == J7_CONST) {
                                v = s0 * c + s1 * (((xn[0][0] + xn[0][1]) + (yn[0][0] + yn[0][1])) + (zn[0][0] + zn[0][1]));
                            } else if constexpr (KIND == J7_VAR) {
                                const T *Wp = a.W + idx;
                                const int64_t n = g.nfield;
                                v = Wp[0] * c;
                                v = fma(Wp[1 * n], xn[0][0], v);
                                v = fma(Wp[2 * n], xn[0][1], v);
                                v = fma(Wp[3 * n], yn[0][0], v);
                                v = fma(Wp[4 * n], yn[0][1], v);
                                v = fma(Wp[5 * n], zn[0][0], v);
                                v = fma(Wp[6 * n], zn[0][1], v);
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
                                v = fma(a.W[idx], s, T(2) * c - pv);
                            } else {  // W25_VAR, J25_VAR
                                const T *Wp = a.W + idx;
                                const int64_t n = g.nfield;
                                T acc = Wp[0] * c;
                                if constexpr (WAVE) acc = fma(T(2), c, acc) - pv;
#pragma unroll
                                for (int d = 0; d < 4; ++d) {
                                    acc = fma(Wp[(3 * d + 1) * n], xn[d][0] + xn[d][1], acc);
                                    acc = fma(Wp[(3 * d + 2) * n], yn[d][0] + yn[d][1], acc);
                                    acc = fma(Wp[(3 * d + 3) * n], zn[d][0] + zn[d][1], acc);
                                }
                                v = acc;
                            }
                            if (zown && xown && Rw::owned(k, ry)) {
                                if (a.trace && z == a.rcv_z) a.trace[(k - 1) * plane_elems + (int64_t)y * g.nx + x] = v;
                                if constexpr (k == B) {
                                    a.out[idx] = v;
                                }
                            }
                            if constexpr (PHASE == PH_A && k < B) {
                                if (zown && xown && Rw::band_store(k, ry)) a.bands[k][idx] = v;
                            }
                        }
                    } else if constexpr (PHASE == PH_B && k < B) {
                        if (Rw::band_load(k, ry) && in) v = a.bands[k][idx];
                    }
                    if constexpr (k == B) {
                        // level B-1 at plane z: the next pass's u^{t-1}
                        if (a.out_prev && in && zown && xown && Rw::owned(B - 1, ry) &&
                            (PHASE != PH_OVL || Rw::owned(B, ry)))
                            a.out_prev[idx] = ring[B - 1][jc][r];
                    } else {
                        ring[k][jc][r] = v;
                    }
                }
            });
            par ^= 1;
        });
    }
}

// ---------------------------------------------------------------- configs
// Per radius: tile of the overlapped / phase-A launch (TX x BY threads, NR
// rows each) and of the phase-B launch (2(B+1)R rows).
template <int R, int B> struct Cfg;
template <int B> struct Cfg<1, B> {
    static constexpr int TX = 64, BY = 8, NR = 4;                 // 64 x 32 region
    static constexpr int BTX = 64, BNR = 2, BBY = (B + 1);        // 64 x 2(B+1)
};
template <int B> struct Cfg<4, B> {
    static constexpr int TX = 64, BY = 8, NR = 3;                 // 64 x 24 region
    static constexpr int BTX = 64, BNR = 3, BBY = 8 * (B + 1) / 3;  // 64 x 2(B+1)R
};

template <typename T, int KIND, int PHASE, int B, int TX, int BY, int NR>
static cudaError_t launch_one(const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int gy) {
    auto kern = blocked_kernel<T, KIND, PHASE, B, TX, BY, NR>;
    constexpr int R = KindTraits<KIND>::R;
    constexpr size_t smem = sizeof(T) * (size_t)B * 2 * (TX + 2 * R) * (BY * NR + 2 * R);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * BY, smem);
    if (per_sm < 1) per_sm = 1;
    constexpr int TXO = TX - 2 * B * R;
    const int gx = (a.g.nx + TXO - 1) / TXO;
    // z chunks: about 3 waves of CTAs, each chunk at least 8*B*R planes
    const int64_t want = (int64_t)num_sms * per_sm * 3;
    const int64_t tiles = (int64_t)gx * gy;
    int nzc = (int)((want + tiles - 1) / tiles);
    const int min_chunk = 8 * B * R;
    if (nzc < 1) nzc = 1;
    if ((a.g.nz + nzc - 1) / nzc < min_chunk) nzc = (a.g.nz + min_chunk - 1) / min_chunk;
    if (nzc < 1) nzc = 1;
    BlockedArgs<T> b = a;
    b.zchunk = (a.g.nz + nzc - 1) / nzc;
    const int gz = (a.g.nz + b.zchunk - 1) / b.zchunk;
    dim3 grid(gx, gy, gz), block(TX, BY, 1);
    kern<<<grid, block, smem, st>>>(b);
    return cudaGetLastError();
}

template <typename T, int KIND, int B>
static cudaError_t launch_levels(const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int scheme) {
    constexpr int R = KindTraits<KIND>::R;
    using C = Cfg<R, B>;
    constexpr int RY = C::BY * C::NR;
    if (scheme == 1) {
        constexpr int WO = RY - 2 * B * R;
        if constexpr (WO > 0) {
            const int gy = (a.g.ny + WO - 1) / WO;
            return launch_one<T, KIND, PH_OVL, B, C::TX, C::BY, C::NR>(a, st, num_sms, gy);
        } else {
            return cudaErrorNotSupported;
        }
    }
    // diamond: phase A then phase B (stream order makes A's bands visible)
    BlockedArgs<T> b = a;
    b.wA = RY;
    const int nA = (a.g.ny + RY - 1) / RY;
    cudaError_t e = launch_one<T, KIND, PH_A, B, C::TX, C::BY, C::NR>(b, st, num_sms, nA);
    if (e != cudaSuccess) return e;
    static_assert(C::BBY * C::BNR == 2 * (B + 1) * R, "phase B rows");
    return launch_one<T, KIND, PH_B, B, C::BTX, C::BBY, C::BNR>(b, st, num_sms, nA + 1);
}

template <typename T, int KIND>
static cudaError_t launch_kind(const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int scheme) {
    constexpr int R = KindTraits<KIND>::R;
    if constexpr (R == 1) {
        switch (a.levels) {
        case 2: return launch_levels<T, KIND, 2>(a, st, num_sms, scheme);
        case 4: return launch_levels<T, KIND, 4>(a, st, num_sms, scheme);
        default: return cudaErrorNotSupported;
        }
    } else {
        switch (a.levels) {
        case 2: return launch_levels<T, KIND, 2>(a, st, num_sms, scheme);
        default: return cudaErrorNotSupported;
        }
    }
}

bool blocked_supported(int kind, int dtype, int levels) {
    if (dtype != 1) return false;  // FP32 only: FP64 sweeps are bound by the FP64 pipe
    const int R = kind_radius(kind);
    if (R == 1) return levels == 2 || levels == 4;
    if (R == 4) return levels == 2;
    return false;
}

int blocked_default_levels(int kind, int dtype) {
    if (dtype != 1) return 1;
    return kind_radius(kind) == 1 ? 4 : 2;
}

int blocked_scratch_levels(int levels) { return levels > 1 ? levels - 1 : 0; }

template <typename T>
cudaError_t launch_blocked(int kind, const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int scheme) {
    if (scheme == 0) scheme = 2;
    if constexpr (sizeof(T) == 4) {
        switch (kind) {
        case J7_CONST: return launch_kind<T, J7_CONST>(a, st, num_sms, scheme);
        case J7_VAR: return launch_kind<T, J7_VAR>(a, st, num_sms, scheme);
        case W25_CONST: return launch_kind<T, W25_CONST>(a, st, num_sms, scheme);
        case W25_VAR: return launch_kind<T, W25_VAR>(a, st, num_sms, scheme);
        case J25_VAR: return launch_kind<T, J25_VAR>(a, st, num_sms, scheme);
        case W25_ALPHA: return launch_kind<T, W25_ALPHA>(a, st, num_sms, scheme);
        default: return cudaErrorInvalidValue;
        }
    } else {
        return cudaErrorNotSupported;
    }
}

template cudaError_t launch_blocked<float>(int, const BlockedArgs<float> &, cudaStream_t, int, int);
template cudaError_t launch_blocked<double>(int, const BlockedArgs<double> &, cudaStream_t, int, int);

}  // namespace stc
