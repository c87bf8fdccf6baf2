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
//    multi-thread wavefront (Sect. 5.1, MWD) is the CTA sharing its SM's
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

// CS: coefficient planes are staged once per pass in a shared-memory ring of
// NCS = (B-1)R + PD + 2 plane slots and reused by all B levels (a plane is
// issued PD steps before level 1 needs it and read last by level B, (B-1)R
// steps later); otherwise each level loads them from global memory / L2.
template <typename T, int KIND, int PHASE, int B, int TX, int BY, int NR, int PD, bool CS = false>
__global__ void __launch_bounds__(TX * BY)
blocked_kernel(const BlockedArgs<T> a) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int NA = KindTraits<KIND>::NARR;
    constexpr int NAB = NA > 0 ? NA : 1;
    constexpr int RY = BY * NR;
    constexpr int RING = 2 * R + 1;
    constexpr int PX = TX + 2 * R;      // shared plane pitch (R pad on each side)
    constexpr int PY = RY + 2 * R;
    constexpr int PLANE = PX * PY;
    constexpr int M0 = (R + 2 + PD + RING - 1) / RING;
    constexpr int NS0 = M0 * RING;      // level-0 plane slots
    static_assert(PHASE != PH_B || RY == 2 * (B + 1) * R, "phase B region is 2(B+1)R rows");
    static_assert(PHASE == PH_B || RY >= 2 * B * R, "tile must hold the trapezoid");
    static_assert(NR <= 32, "row masks");
    // coefficient loads are issued one level ahead when the double buffer
    // fits in registers; otherwise at the start of each level
    constexpr bool CST = CS && NA > 0;
    constexpr bool PREF = !CST && NA * NR <= 28;
    constexpr int NCS = (B - 1) * R + PD + 2;
    constexpr int CPL = NAB * RY * TX;    // one staged coefficient plane
    using Rw = Rows<PHASE, B, R, RY>;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *s0buf = reinterpret_cast<T *>(smem_raw);        // [NS0][PLANE] level 0
    T *sbuf = s0buf + NS0 * PLANE;                      // [B-1][2][PLANE] levels 1..B-1
    T *cbuf = sbuf + 2 * (B - 1) * PLANE;               // CST: [NCS][NA][RY][TX]
    (void)cbuf;

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
    const int sy = (int)g.sy;
    const int qs = z0 - B * R, qe = z1 + B * R;
    const int64_t plane_elems = (int64_t)g.nx * g.ny;

    // ---- per-thread constants: copy plan of level 0 (rows ty + i BY of
    // column tx, zero outside the padded array) and masks of own rows
    const bool xmem = x >= -R && x < g.nx + R;
    uint32_t cmask = 0;      // copy rows inside the padded array
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int y = Y0 + ty + i * BY;
        if (xmem && y >= -R && y < g.ny + R) cmask |= 1u << i;
    }
    const int coff0 = (Y0 + ty + R) * sy + (x + R);     // padded in-plane offset of copy row 0
    uint32_t ymask = 0;      // own rows inside the interior (and the column inside)
#pragma unroll
    for (int jr = 0; jr < NR; ++jr) {
        const int y = Y0 + ty * NR + jr;
        if (xin && y >= 0 && y < g.ny) ymask |= 1u << jr;
    }
    const int pofs0 = (Y0 + ty * NR + R) * sy + (x + R);  // padded in-plane offset of own row 0

    uint32_t imask = 0;      // copy rows inside the interior (coefficient staging)
#pragma unroll
    for (int i = 0; i < NR; ++i) {
        const int y = Y0 + ty + i * BY;
        if (xin && y >= 0 && y < g.ny) imask |= 1u << i;
    }
    // coefficient plane p into ring slot (p mod NCS)
    auto issue_coef = [&](int p) {
        if constexpr (CST) {
            if (p < 0 || p >= g.nz) return;
            T *d = cbuf + cmod(p, NCS) * CPL + ty * TX + tx;
            const T *src = a.W + (int64_t)(p + R) * g.sz + coff0;
#pragma unroll
            for (int t = 0; t < NA; ++t)
#pragma unroll
                for (int i = 0; i < NR; ++i)
                    if (imask & (1u << i))
                        cp_async<sizeof(T)>(d + t * RY * TX + i * BY * TX, src + t * g.nfield + i * BY * sy);
        }
    };
    auto issue0 = [&](int q, T *slot) {
        const bool qmem = q >= -R && q < g.nz + R;
        const T *pb = a.u + (qmem ? (int64_t)(q + R) * g.sz : 0) + coff0;
        T *d = slot + (ty + R) * PX + tx + R;
#pragma unroll
        for (int i = 0; i < NR; ++i) {
            const bool ok = qmem && (cmask & (1u << i));
            cp_async_zfill<sizeof(T)>(d + i * BY * PX, ok ? (const void *)(pb + i * BY * sy) : (const void *)a.u, ok);
        }
    };

    T ring[B][RING][NR];
#pragma unroll
    for (int k = 0; k < B; ++k)
#pragma unroll
        for (int i = 0; i < RING; ++i)
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) ring[k][i][jr] = T(0);

    // u^{t-1} of level 1 (second order), one step ahead
    T preP[NR];
    auto load_prev = [&](int z) {
        const bool zin = z >= 0 && z < g.nz;
        const int64_t zo = (int64_t)(z + R) * g.sz + pofs0;
#pragma unroll
        for (int jr = 0; jr < NR; ++jr)
            preP[jr] = (zin && (ymask & (1u << jr))) ? a.u_prev[zo + jr * sy] : T(0);
    };
    // coefficients of level k at plane z for own rows
    T cf[NAB][NR], cfn[NAB][NR];
#pragma unroll
    for (int t = 0; t < NAB; ++t)
#pragma unroll
        for (int jr = 0; jr < NR; ++jr) { cf[t][jr] = T(0); cfn[t][jr] = T(0); }
    auto load_cf = [&](int z) {
        if constexpr (NA > 0) {
            if (z < 0 || z >= g.nz) return;
            const int64_t zo = (int64_t)(z + R) * g.sz + pofs0;
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) {
                if (!(ymask & (1u << jr))) continue;
#pragma unroll
                for (int t = 0; t < NA; ++t) cfn[t][jr] = a.W[zo + jr * sy + t * g.nfield];
            }
        }
    };

#pragma unroll
    for (int i = 0; i < PD; ++i) {
        if (qs + i < qe) {
            issue0(qs + i, s0buf + i * PLANE);
            issue_coef(qs + i - R);
        }
        cp_async_commit();
    }
    if constexpr (WAVE) load_prev(qs - R);

    const T s0 = T(a.s.c[0]), s1 = T(a.s.c[1]), s2 = T(a.s.c[2]);
    const T s3 = T(a.s.c[3]), s4 = T(a.s.c[4]);
    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4;

    int par = 0, blk = 0;
    for (int qb = qs; qb < qe; qb += RING) {
        T *const slots0 = s0buf + blk * RING * PLANE;
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            const int q = qb + j;
            if (q >= qe) return;
            T curP[NR];
#pragma unroll
            for (int jr = 0; jr < NR; ++jr) curP[jr] = preP[jr];
            if constexpr (WAVE) {
                if (q + 1 < qe) load_prev(q + 1 - R);
            }
            if constexpr (NA > 0 && PREF) load_cf(q - R);   // level 1 of this step
            {
                T *dst = slots0 + (j + PD) * PLANE;
                if (j + PD >= NS0 - blk * RING) dst -= NS0 * PLANE;
                if (q + PD < qe) {
                    issue0(q + PD, dst);
                    issue_coef(q + PD - R);
                }
            }
            cp_async_commit();
            // centre planes of levels 1..B-1 (inputs of levels 2..B)
            static_for<B - 1>([&](auto kk) {
                constexpr int k = decltype(kk)::value + 1;       // level whose plane is written
                if (q < qs + 2 * (k + 1) * R) return;
                T *buf = sbuf + ((k - 1) * 2 + par) * PLANE + (ty * NR + R) * PX + tx + R;
                constexpr int jc = cmod(j - (k + 1) * R, RING);
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) buf[jr * PX] = ring[k][jc][jr];
            });
            cp_async_wait<PD>();
            __syncthreads();
            // level-0 front
            {
                const T *sq = slots0 + j * PLANE + (ty * NR + R) * PX + tx + R;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) ring[0][j][jr] = sq[jr * PX];
            }
            // levels 1..B
            static_for<B>([&](auto kk) {
                constexpr int k = decltype(kk)::value + 1;
                if (q < qs + 2 * k * R) return;
                const int z = q - k * R;
                const bool zin = z >= 0 && z < g.nz;
                const bool zown = z >= z0 && z < z1;
                // coefficients: this level's arrived, prefetch the next level's
                if constexpr (CST) {
                    if (z >= 0 && z < g.nz) {
                        const T *cs = cbuf + cmod(z, NCS) * CPL + (ty * NR) * TX + tx;
#pragma unroll
                        for (int t = 0; t < NA; ++t)
#pragma unroll
                            for (int jr = 0; jr < NR; ++jr) cf[t][jr] = cs[t * RY * TX + jr * TX];
                    }
                } else if constexpr (NA > 0) {
                    if constexpr (!PREF) load_cf(z);
#pragma unroll
                    for (int t = 0; t < NA; ++t)
#pragma unroll
                        for (int jr = 0; jr < NR; ++jr) cf[t][jr] = cfn[t][jr];
                    if constexpr (PREF && k < B) load_cf(z - R);
                }
                const T *sp;
                if constexpr (k == 1) {
                    T *p0 = slots0 + (j - R) * PLANE;
                    if (j - R < -blk * RING) p0 += NS0 * PLANE;
                    sp = p0;
                } else {
                    sp = sbuf + ((k - 2) * 2 + par) * PLANE;
                }
                const T *rowp = sp + (ty * NR + R) * PX + tx + R;
                constexpr int jc = cmod(j - k * R, RING);
                const int64_t zoff = (int64_t)(z + R) * g.sz + pofs0;
#pragma unroll
                for (int jr = 0; jr < NR; ++jr) {
                    const int ry = ty * NR + jr;
                    const bool in = zin && (ymask & (1u << jr));
                    T v = T(0);
                    // Overlapped / phase-A tiles compute every row at every level
                    // without a branch: rows outside the level's valid band hold
                    // values that only feed rows that are never stored (the valid
                    // band shrinks by R per level); points outside the interior
                    // take the zero Dirichlet value by a select.  Phase-B tiles
                    // compute their growing band and load the rest from the bands.
                    if (PHASE != PH_B || Rw::computed(k, ry)) {
                        if (PHASE != PH_B || in) {
                            const T *cp = rowp + jr * PX;
                            const T c = ring[k - 1][jc][jr];
                            T xn[R][2], yn[R][2], zn[R][2];
#pragma unroll
                            for (int d = 1; d <= R; ++d) {
                                xn[d - 1][0] = cp[-d];
                                xn[d - 1][1] = cp[d];
                                if (jr - d >= 0) yn[d - 1][0] = ring[k - 1][jc][jr - d];
                                else yn[d - 1][0] = cp[-d * PX];
                                if (jr + d < NR) yn[d - 1][1] = ring[k - 1][jc][jr + d];
                                else yn[d - 1][1] = cp[d * PX];
                                zn[d - 1][0] = ring[k - 1][cmod(j - k * R - d, RING)][jr];
                                zn[d - 1][1] = ring[k - 1][cmod(j - k * R + d, RING)][jr];
                            }
                            T pv = T(0);
                            if constexpr (WAVE) {
                                if constexpr (k == 1) pv = curP[jr];
                                else pv = ring[k - 2][jc][jr];
                            }
                            (void)pv;
                            constexpr int CO = (KIND == W25_ALPHA) ? 0 : 0;
                            (void)CO;
                            if constexpr (KIND == J7_CONST) {
                                v = s0 * c + s1 * (((xn[0][0] + xn[0][1]) + (yn[0][0] + yn[0][1])) + (zn[0][0] + zn[0][1]));
                            } else if constexpr (KIND == J7_VAR) {
                                v = cf[0][jr] * c;
                                v = fma(cf[1][jr], xn[0][0], v);
                                v = fma(cf[2][jr], xn[0][1], v);
                                v = fma(cf[3][jr], yn[0][0], v);
                                v = fma(cf[4][jr], yn[0][1], v);
                                v = fma(cf[5][jr], zn[0][0], v);
                                v = fma(cf[6][jr], zn[0][1], v);
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
                                v = fma(cf[0][jr], s, T(2) * c - pv);
                            } else {  // W25_VAR, J25_VAR
                                T acc = cf[0][jr] * c;
                                if constexpr (WAVE) acc = fma(T(2), c, acc) - pv;
#pragma unroll
                                for (int d = 0; d < 4; ++d) {
                                    acc = fma(cf[3 * d + 1][jr], xn[d][0] + xn[d][1], acc);
                                    acc = fma(cf[3 * d + 2][jr], yn[d][0] + yn[d][1], acc);
                                    acc = fma(cf[3 * d + 3][jr], zn[d][0] + zn[d][1], acc);
                                }
                                v = acc;
                            }
                            if constexpr (PHASE != PH_B) v = in ? v : T(0);
                            if (in && zown && xown && Rw::computed(k, ry)) {
                                if (Rw::owned(k, ry)) {
                                    if (z == a.rcv_z && a.trace)
                                        a.trace[(k - 1) * plane_elems + (int64_t)(Y0 + ry) * g.nx + x] = v;
                                    if constexpr (k == B)
                                        if (dbg_store_ok(a.dbg, g, zoff + jr * sy)) a.out[zoff + jr * sy] = v;
                                }
                                if constexpr (PHASE == PH_A && k < B) {
                                    if (Rw::band_store(k, ry)) a.bands[k][zoff + jr * sy] = v;
                                }
                            }
                        }
                    } else if constexpr (PHASE == PH_B && k < B) {
                        if (Rw::band_load(k, ry) && in) v = a.bands[k][zoff + jr * sy];
                    }
                    if constexpr (k == B) {
                        // level B-1 at plane z: the next pass's u^{t-1}
                        if (a.out_prev && in && zown && xown && Rw::owned(B - 1, ry) &&
                            (PHASE != PH_OVL || Rw::owned(B, ry)))
                            if (dbg_store_ok(a.dbg, g, zoff + jr * sy)) a.out_prev[zoff + jr * sy] = ring[B - 1][jc][jr];
                    } else {
                        ring[k][jc][jr] = v;
                    }
                }
            });
            par ^= 1;
        });
        blk = (blk + 1 == M0) ? 0 : blk + 1;
    }
}

template <typename T, int KIND, int B, int TX, int BY, int NR, int PD, bool CS = false>
constexpr size_t blocked_smem() {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int RING = 2 * R + 1;
    constexpr int M0 = (R + 2 + PD + RING - 1) / RING;
    constexpr int NA = KindTraits<KIND>::NARR;
    constexpr size_t cs = (CS && NA > 0) ? (size_t)((B - 1) * R + PD + 2) * NA * BY * NR * TX : 0;
    return sizeof(T) * ((size_t)(M0 * RING + 2 * (B - 1)) * (TX + 2 * R) * (BY * NR + 2 * R) + cs);
}

// ---------------------------------------------------------------- configs
// Per element size, radius, block depth and coefficient staging: tile of the
// overlapped / phase-A launch (TX x BY threads, NR rows each) and of the
// phase-B launch (2(B+1)R rows).  With staged coefficients (CS) the region is
// kept small enough for the coefficient ring to fit shared memory.
template <int WORD, int R, int B, bool CS> struct Cfg;
template <int B> struct Cfg<4, 1, B, false> {
    static constexpr int TX = 64, BY = 8, NR = 4;                 // 64 x 32 region
    static constexpr int BTX = 64, BNR = 2, BBY = (B + 1);        // 64 x 2(B+1)
};
template <int B> struct Cfg<4, 1, B, true> {
    static constexpr int TX = (B <= 3 ? 64 : 32), BY = 4, NR = 4; // 64 x 16 (32 x 16 for B = 4)
    static constexpr int BTX = TX, BNR = 2, BBY = (B + 1);
};
template <int B> struct Cfg<4, 4, B, false> {
    static constexpr int TX = 64, BY = 8, NR = 3;                 // 64 x 24 region
    static constexpr int BTX = 64, BNR = 3, BBY = 8 * (B + 1) / 3;  // 64 x 2(B+1)R
};
template <int B> struct Cfg<4, 4, B, true> : Cfg<4, 4, B, false> {};
template <int B, bool CS> struct Cfg<8, 1, B, CS> {               // FP64: 256-thread tiles
    static constexpr int TX = 32, BY = 8, NR = 2;                 // 32 x 16 region
    static constexpr int BTX = 32, BNR = 2, BBY = (B + 1);
};

template <typename T, int KIND, int PHASE, int B, int TX, int BY, int NR, bool CS>
static cudaError_t launch_one(const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int gy) {
    constexpr int PD = 2;
    auto kern = blocked_kernel<T, KIND, PHASE, B, TX, BY, NR, PD, CS>;
    constexpr int R = KindTraits<KIND>::R;
    constexpr size_t smem = blocked_smem<T, KIND, B, TX, BY, NR, PD, CS>();
    static_assert(smem <= 227 * 1024, "shared memory per CTA");
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, TX * BY, smem);
    if (per_sm < 1) per_sm = 1;
    constexpr int TXO = TX - 2 * B * R;
    const int gx = (a.g.nx + TXO - 1) / TXO;
    // z chunks: enough CTAs for one to two waves; every chunk recomputes a
    // ramp of 2BR planes, so chunks are at least 16BR (and 32) planes long
    const int64_t want = (int64_t)num_sms * per_sm;
    const int64_t tiles = (int64_t)gx * gy;
    int nzc = (int)((want + tiles - 1) / tiles);
    const int min_chunk = 16 * B * R > 32 ? 16 * B * R : 32;
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
    constexpr bool CS = KindTraits<KIND>::NARR > 0 && R == 1;   // stage the 7 coefficient planes
    using C = Cfg<(int)sizeof(T), R, B, CS>;
    constexpr int RY = C::BY * C::NR;
    if (scheme == 1) {
        constexpr int WO = RY - 2 * B * R;
        if constexpr (WO > 0) {
            const int gy = (a.g.ny + WO - 1) / WO;
            return launch_one<T, KIND, PH_OVL, B, C::TX, C::BY, C::NR, CS>(a, st, num_sms, gy);
        } else {
            return cudaErrorNotSupported;
        }
    }
    // diamond: phase A then phase B (stream order makes A's bands visible)
    BlockedArgs<T> b = a;
    b.wA = RY;
    const int nA = (a.g.ny + RY - 1) / RY;
    cudaError_t e = launch_one<T, KIND, PH_A, B, C::TX, C::BY, C::NR, CS>(b, st, num_sms, nA);
    if (e != cudaSuccess) return e;
    static_assert(C::BBY * C::BNR == 2 * (B + 1) * R, "phase B rows");
    return launch_one<T, KIND, PH_B, B, C::BTX, C::BBY, C::BNR, CS>(b, st, num_sms, nA + 1);
}

template <typename T, int KIND>
static cudaError_t launch_kind(const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int scheme) {
    constexpr int R = KindTraits<KIND>::R;
    if constexpr (R == 1) {
        switch (a.levels) {
        case 2: return launch_levels<T, KIND, 2>(a, st, num_sms, scheme);
        case 3: return launch_levels<T, KIND, 3>(a, st, num_sms, scheme);
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
    const int R = kind_radius(kind);
    if (dtype != 1) return R == 1 && levels == 2;  // FP64: 7-point kinds, two levels per pass
    if (R == 1) return levels >= 2 && levels <= 4;
    if (R == 4) return levels == 2;
    return false;
}

// Default block depth per kind and dtype (measured, 512^3): 1 where the
// plain streaming sweep is faster.
int blocked_default_levels(int kind, int dtype) {
    (void)kind;
    (void)dtype;
    return 1;
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
        switch (kind) {
        case J7_CONST:
            return a.levels == 2 ? launch_levels<T, J7_CONST, 2>(a, st, num_sms, scheme) : cudaErrorNotSupported;
        case J7_VAR:
            return a.levels == 2 ? launch_levels<T, J7_VAR, 2>(a, st, num_sms, scheme) : cudaErrorNotSupported;
        default: return cudaErrorNotSupported;
        }
    }
}

template cudaError_t launch_blocked<float>(int, const BlockedArgs<float> &, cudaStream_t, int, int);
template cudaError_t launch_blocked<double>(int, const BlockedArgs<double> &, cudaStream_t, int, int);

}  // namespace stc
