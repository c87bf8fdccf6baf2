// blk25_impl.cuh -- temporally blocked pass of the 13-array 25-point kinds
// (Fig. 1d structure, R = 4): two time levels per sweep over HBM, FP32.
// Included by plainv_f32.cu (TMA / mbarrier helpers, tensor maps, the
// bounded-wait counter of that translation unit).
//
// The z wavefront of Sect. 4.1 with two levels: when level-0 plane q has
// arrived, level 1 updates plane q - R and level 2 plane q - 2R (frontline
// slope -1/R).  A CTA owns a 64 x 16 tile of every plane; level 1 is computed
// on the tile with a halo of R points on each side (72 x 24: the y and x
// extent level 2 reads), from level 0 on the tile with a halo of 2R (80 x 32).
// All three live in shared memory as plane rings:
//   level 0   11 slots (the 2R+1 planes level 1 reads, two planes in flight),
//             each brought by one bulk tensor copy (zero fill outside the
//             padded array), with u^{t-1} of level 1's plane beside it
//             (3 slots) for the second-order kind;
//   level 1   9 slots (the 2R+1 planes level 2 reads), written by the CTA.
// Every neighbour, in x, y and z, is an aligned 16-byte shared load (4 points
// per thread-vector).  The 13 coefficient vectors of a point are read from
// global memory at the point: level 1 reads them for its halo'd tile, level 2
// R steps later for the owned tile -- the second read is meant to hit L2
// (all tiles of a plane march z together: the grid covers the lattice's x-y
// extent with resident CTAs).  HBM then carries u^t, u^{t-1} and the 13
// arrays once and the two written levels once per two time steps.
// Points outside the interior hold the zero Dirichlet value at level 1 (their
// value is selected to zero; their coefficients are not read).
// Level 2 and, for the next pass's u^{t-1}, level 1 are written for the owned
// points; the receiver trace of both levels as well.
//
// Measured (512^3, FP32, T = 64): 71 GLUP/s for W25_VAR and 75 for J25_VAR,
// against 105 and 114 for the one-level TMA sweep, so it is not the default.
// ncu (384^3, one pass): DRAM 36.5 bytes per update (34 algorithmic, 64 for
// the one-level sweep) with an L2 hit rate of 50% -- the coefficient re-read
// is served by L2 -- but the 196 KB of plane rings leave one 256-thread CTA
// per SM: 8 warps, 28% issue activity, long-scoreboard and barrier stalls.
// A warp-specialised form (14 level-1 and 8 level-2 warps working on the
// same step, one barrier per step) was measured slower (42 GLUP/s): 704
// threads leave 80 registers per thread and the coefficient vectors spill.
#pragma once
#include "blocked.cuh"

namespace stc {

namespace b25 {
constexpr int R = 4, V = 4;
constexpr int TXO = 64, TYO = 16;              // owned tile
constexpr int TX1 = TXO + 2 * R, TY1 = TYO + 2 * R;   // level-1 tile (72 x 24)
constexpr int TX0 = TXO + 4 * R, TY0 = TYO + 4 * R;   // level-0 tile (80 x 32)
constexpr int NV1 = TX1 / V, NP1 = NV1 * TY1;  // level-1 vectors per row / per plane (18, 432)
constexpr int NVO = TXO / V, NPO = NVO * TYO;  // owned vectors per row / per plane (16, 256)
constexpr int NT = 256;                        // threads
constexpr int PD = 2;                          // level-0 planes in flight
constexpr int NS0 = 2 * R + 1 + PD;            // level-0 slots
constexpr int NSP = PD + 1;                    // u^{t-1} slots
constexpr int NS1 = 2 * R + 1;                 // level-1 slots
constexpr int P0 = TX0 * TY0, P1 = TX1 * TY1;  // plane sizes (floats)
static_assert((P0 * 4) % 128 == 0 && (P1 * 4) % 128 == 0, "128-byte aligned planes");
constexpr size_t smem_of(bool wave) {
    return 4 * ((size_t)NS0 * P0 + (wave ? (size_t)NSP * P1 : 0) + (size_t)NS1 * P1) + 8 * NS0 + 16 + 128;
}
}  // namespace b25

template <int KIND>
__global__ void __launch_bounds__(b25::NT, 1)
blk25_kernel(const BlockedArgs<float> a, const __grid_constant__ CUtensorMap tm_u,
             const __grid_constant__ CUtensorMap tm_p) {
    using namespace b25;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const s0 = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *const sp = s0 + NS0 * P0;                      // u^{t-1} slots (wave kind)
    float *const s1 = sp + (WAVE ? NSP * P1 : 0);         // level-1 slots
    uint64_t *const bars = reinterpret_cast<uint64_t *>(s1 + NS1 * P1);
    volatile int &abort_word = *reinterpret_cast<volatile int *>(bars + NS0);

    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const int xo = blockIdx.x * TXO + R, yo = blockIdx.y * TYO + R;   // padded origin of the owned tile
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int qs = z0 - 2 * R, qe = z1 + 2 * R;            // level-0 planes this chunk reads
    const int64_t sz = g.sz, sy = g.sy, nf = g.nfield;
    const int64_t plane_elems = (int64_t)g.nx * g.ny;

    // level-1 vectors of this thread: k = tid and tid + NT (while < NP1)
    constexpr int NK1 = (NP1 + NT - 1) / NT;
    int r1[NK1], c1[NK1];           // level-1 tile row, column
    bool in1[NK1], act1[NK1];       // interior point vector; computed by this thread
    int64_t g1[NK1];                // in-plane padded offset
#pragma unroll
    for (int u = 0; u < NK1; ++u) {
        const int k = tid + u * NT;
        act1[u] = k < NP1;
        r1[u] = act1[u] ? k / NV1 : 0;
        c1[u] = act1[u] ? (k % NV1) * V : 0;
        const int py = yo - R + r1[u], px = xo - R + c1[u];
        in1[u] = act1[u] && py >= R && py < g.ny + R && px >= R && px < g.nx + R;
        g1[u] = in1[u] ? (int64_t)py * sy + px : 0;
    }
    // owned vector of this thread (level 2)
    const int r2 = tid / NVO, c2 = (tid % NVO) * V;
    const int py2 = yo + r2, px2 = xo + c2;
    const bool in2 = py2 < g.ny + R && px2 < g.nx + R;
    const int64_t g2 = in2 ? (int64_t)py2 * sy + px2 : 0;
    // owned level-1 vectors (for out_prev and the level-1 trace)
    bool own1[NK1];
#pragma unroll
    for (int u = 0; u < NK1; ++u)
        own1[u] = in1[u] && r1[u] >= R && r1[u] < R + TYO && c1[u] >= R && c1[u] < R + TXO;

    bool bad = false;
    int last_issued = qs - 1;
    const int wlim = pv::wait_limit_of(a.wait_limit);
    auto issue = [&](int q) {
        if (bad) return;
        const int s = (q - qs) % NS0;
        last_issued = q;
        pv::mbar_expect_tx(&bars[s], (uint32_t)(4 * (P0 + (WAVE ? P1 : 0))));
        pv::tma_load_3d(s0 + s * P0, &tm_u, xo - 2 * R, yo - 2 * R, q + R, &bars[s]);
        if constexpr (WAVE)   // u^{t-1} of level 1's plane q - R, level-1 tile
            pv::tma_load_3d(sp + ((q - qs) % NSP) * P1, &tm_p, xo - R, yo - R, q, &bars[s]);
    };
    if (tid < NS0) pv::mbar_init(&bars[tid], 1);
    if (tid == 0) abort_word = 0;
    pv::mbar_init_fence();
    __syncthreads();
    if (tid == 0)
        for (int i = 0; i < PD && qs + i < qe; ++i) issue(qs + i);

    // stencil of the 13-array kinds at a 4-point vector: tile row r, column
    // c of planes of width W; plane_at(d) is the plane d planes from the centre
    auto update = [&](auto plane_at, int W, int r, int c, const float4 (&cf)[13], float4 prev) -> float4 {
        const float *C = plane_at(0) + r * W + c;
        const float4 cv = *reinterpret_cast<const float4 *>(C);
        const float4 lv = *reinterpret_cast<const float4 *>(C - V);
        const float4 rv = *reinterpret_cast<const float4 *>(C + V);
        const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
        const float ll[4] = {lv.x, lv.y, lv.z, lv.w};
        const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
        float acc[4];
        const float c0[4] = {cf[0].x, cf[0].y, cf[0].z, cf[0].w};
        const float pr[4] = {prev.x, prev.y, prev.z, prev.w};
        (void)pr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i] = c0[i] * cc[i];
            if constexpr (WAVE) acc[i] = fma(2.0f, cc[i], acc[i]) - pr[i];
        }
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            const float4 yu = *reinterpret_cast<const float4 *>(C - d * W);
            const float4 yd = *reinterpret_cast<const float4 *>(C + d * W);
            const float4 zd = *reinterpret_cast<const float4 *>(plane_at(-d) + r * W + c);
            const float4 zu = *reinterpret_cast<const float4 *>(plane_at(d) + r * W + c);
            const float yuu[4] = {yu.x, yu.y, yu.z, yu.w}, ydd[4] = {yd.x, yd.y, yd.z, yd.w};
            const float zdd[4] = {zd.x, zd.y, zd.z, zd.w}, zuu[4] = {zu.x, zu.y, zu.z, zu.w};
            const float4 wx = cf[3 * d - 2], wy = cf[3 * d - 1], wz = cf[3 * d];
            const float wxx[4] = {wx.x, wx.y, wx.z, wx.w}, wyy[4] = {wy.x, wy.y, wy.z, wy.w};
            const float wzz[4] = {wz.x, wz.y, wz.z, wz.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float xl = i - d >= 0 ? cc[i - d] : ll[i - d + 4];
                const float xr = i + d < 4 ? cc[i + d] : rr[i + d - 4];
                acc[i] = fma(wxx[i], xl + xr, acc[i]);
                acc[i] = fma(wyy[i], yuu[i] + ydd[i], acc[i]);
                acc[i] = fma(wzz[i], zdd[i] + zuu[i], acc[i]);
            }
        }
        return make_float4(acc[0], acc[1], acc[2], acc[3]);
    };
    auto load_cf = [&](float4 (&cf)[13], int64_t off, bool on) {
#pragma unroll
        for (int t = 0; t < 13; ++t)
            cf[t] = on ? __ldg(reinterpret_cast<const float4 *>(a.W + t * nf + off)) : make_float4(0.f, 0.f, 0.f, 0.f);
    };

    bool stop = false;
    for (int q = qs; q < qe && !stop; ++q) {
        const int pc1 = q - R, pc2 = q - 2 * R;   // planes of level 1 and 2 in this step
        const bool l1on = q >= qs + 2 * R && (unsigned)pc1 < (unsigned)g.nz;
        const bool l2on = q >= qs + 4 * R;        // pc2 in [z0, z1)
        // coefficients, issued before the wait: level 2 (owned vector) and
        // the first level-1 vector
        float4 cfa[13], cf2[13];
        load_cf(cf2, (int64_t)(pc2 + R) * sz + g2, l2on && in2);
        load_cf(cfa, (int64_t)(pc1 + R) * sz + g1[0], l1on && in1[0]);
        bad |= !pv::mbar_wait_or_abort(&bars[(q - qs) % NS0], (uint32_t)(((q - qs) / NS0) & 1), wlim, &abort_word);
        if ((q - qs) % 8 == 7) stop = __syncthreads_or(bad);
        else __syncthreads();
        if (tid == 0 && q + PD < qe) issue(q + PD);
        // ---- level 1 at plane pc1 (level-1 tile), into level-1 slot of pc1
        auto l0_at = [&](int d) -> const float * {
            return s0 + ((q - R + d - qs + NS0 * 4) % NS0) * P0;   // level-0 plane pc1 + d
        };
        float *const l1_out = s1 + ((pc1 - qs + NS1 * 4) % NS1) * P1;
        const float *const upl = sp + ((q - qs) % NSP) * P1;
#pragma unroll
        for (int u = 0; u < NK1; ++u) {
            if (!act1[u]) continue;
            float4 cf[13];
            if (u == 0) {
#pragma unroll
                for (int t = 0; t < 13; ++t) cf[t] = cfa[t];
            } else {
                load_cf(cf, (int64_t)(pc1 + R) * sz + g1[u], l1on && in1[u]);
            }
            float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (WAVE) prev = *reinterpret_cast<const float4 *>(upl + r1[u] * TX1 + c1[u]);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (l1on && in1[u]) v = update(l0_at, TX0, r1[u] + R, c1[u] + R, cf, prev);
            *reinterpret_cast<float4 *>(l1_out + r1[u] * TX1 + c1[u]) = v;
            if (own1[u] && (unsigned)pc1 - (unsigned)z0 < (unsigned)(z1 - z0)) {
                const int64_t o = (int64_t)(pc1 + R) * sz + g1[u];
                if (a.out_prev && dbg_store_ok(a.dbg, g, o, V)) *reinterpret_cast<float4 *>(a.out_prev + o) = v;
                if (a.trace && pc1 == a.rcv_z) {
                    float *tr = a.trace + (int64_t)(yo - R + r1[u] - R) * g.nx + (xo - R + c1[u] - R);
                    tr[0] = v.x; tr[1] = v.y; tr[2] = v.z; tr[3] = v.w;
                }
            }
        }
        __syncthreads();
        // ---- level 2 at plane pc2 (owned tile): level-1 planes pc2-R..pc2+R
        if (l2on && in2) {
            auto l1_at = [&](int d) -> const float * { return s1 + ((pc2 + d - qs + NS1 * 4) % NS1) * P1; };
            float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
            if constexpr (WAVE)   // level 0 at plane pc2, the owned point (tile offset 2R)
                prev = *reinterpret_cast<const float4 *>(s0 + ((pc2 - qs) % NS0) * P0 + (r2 + 2 * R) * TX0 + c2 + 2 * R);
            const float4 v = update(l1_at, TX1, r2 + R, c2 + R, cf2, prev);
            const int64_t o = (int64_t)(pc2 + R) * sz + g2;
            if (dbg_store_ok(a.dbg, g, o, V)) *reinterpret_cast<float4 *>(a.out + o) = v;
            if (a.trace && pc2 == a.rcv_z) {
                float *tr = a.trace + plane_elems + (int64_t)(py2 - R) * g.nx + (px2 - R);
                tr[0] = v.x; tr[1] = v.y; tr[2] = v.z; tr[3] = v.w;
            }
        }
    }
    if (__syncthreads_or(bad) && tid == 0) {
        for (int qq = max(last_issued - PD + 1, qs); qq <= last_issued; ++qq)
            pv::mbar_wait(&bars[(qq - qs) % NS0], (uint32_t)(((qq - qs) / NS0) & 1), wlim);
        atomicAdd(&g_wait_timeouts, 1u);
    }
}

// Whether the two-level pass serves the plan: FP32, 13-array kinds, 2
// levels, whole 4-point vectors along x, planes below 2^30 points.
inline bool blk25_supported(int kind, int levels, const Geom &g) {
    return (kind == W25_VAR || kind == J25_VAR) && levels == 2 && g.nx % 4 == 0 &&
           (int64_t)g.px * g.py < ((int64_t)1 << 30);
}

// Resources (as stencil_pass_info reports them).
inline bool blk25_info(int kind, int64_t *info) {
    using namespace b25;
    if (kind != W25_VAR && kind != J25_VAR) return false;
    info[0] = (int64_t)smem_of(kind == W25_VAR);
    info[1] = NT;
    info[2] = TX1;
    info[3] = TY1;
    info[4] = TXO;
    info[5] = TYO;
    return true;
}

inline cudaError_t launch_blk25(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms) {
    using namespace b25;
    const bool wave = kind == W25_VAR;
    CUtensorMap tm_u, tm_p;
    memset(&tm_u, 0, sizeof(tm_u));
    memset(&tm_p, 0, sizeof(tm_p));
    cudaError_t e = pv::make_tmap(&tm_u, a.u, 4, a.g, TX0, TY0);
    if (e == cudaSuccess && wave) e = pv::make_tmap(&tm_p, a.u_prev, 4, a.g, TX1, TY1);
    if (e != cudaSuccess) return e;
    const size_t smem = smem_of(wave);
    auto kern = wave ? blk25_kernel<W25_VAR> : blk25_kernel<J25_VAR>;
    static_assert(smem_of(true) <= 227 * 1024, "shared memory per CTA");
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, NT, smem);
    if (per_sm < 1) per_sm = 1;
    const int gx = (a.g.nx + TXO - 1) / TXO, gy = (a.g.ny + TYO - 1) / TYO;
    // z chunks: minimise (waves of resident CTAs) x (planes per chunk with
    // the 4R planes a chunk re-reads)
    const int64_t resident = (int64_t)num_sms * per_sm, tiles = (int64_t)gx * gy;
    int best = 1;
    double best_cost = 1e300;
    for (int nzc = 1; nzc <= a.g.nz; ++nzc) {
        const int chunk = (a.g.nz + nzc - 1) / nzc;
        if (nzc > 1 && chunk < 16 * R) break;
        const int64_t ctas = tiles * ((a.g.nz + chunk - 1) / chunk);
        const double cost = (double)((ctas + resident - 1) / resident) * (chunk + 4 * R);
        if (cost < best_cost * 0.999) { best_cost = cost; best = nzc; }
    }
    BlockedArgs<float> b = a;
    b.zchunk = (a.g.nz + best - 1) / best;
    dim3 grid(gx, gy, (a.g.nz + b.zchunk - 1) / b.zchunk), block(NT, 1, 1);
    kern<<<grid, block, smem, st>>>(b, tm_u, tm_p);
    return cudaGetLastError();
}

}  // namespace stc
