// blk25_impl.cuh -- temporally blocked pass of the 13-array 25-point kinds
// (Fig. 1d structure, R = 4) and of the constant wave (Fig. 1e form): two
// time levels per sweep over HBM, FP32.
// Included by plainv_f32.cu (TMA / mbarrier helpers, tensor maps, the
// bounded-wait counter of that translation unit).
//
// The z wavefront of Sect. 4.1 with two levels: when level-0 plane q has
// arrived, level 1 updates plane q - R and level 2 plane q - 2R - 1 (one
// plane behind level 1's output, so the two levels of a step need no
// barrier between them).  A CTA owns a 64 x 16 tile of every plane; level 1
// is computed on the tile with a halo of R points on each side (72 x 24: the
// y and x extent level 2 reads), from level 0 on the tile with a halo of 2R
// (80 x 32).  The warps split by level: 14 warps update one level-1 vector
// (4 points) each, 8 warps one owned level-2 vector each, and all meet at
// one barrier per step.  The levels live in shared memory as plane rings:
//   level 0   2R + 2 + PD slots (the 2R + 1 planes level 1 reads, the
//             plane level 2 takes as u^{t-1}, PD planes in flight: 1, 2 for
//             the constant wave), each brought by one bulk tensor copy (zero
//             fill outside the padded array), with u^{t-1} of level 1's
//             plane beside it (PD + 1 slots) for the second-order kinds;
//   level 1   2R + 2 slots (the 2R + 1 planes level 2 reads and the one
//             level 1 writes), written by the CTA.
// Every neighbour, in x, y and z, is an aligned 16-byte shared load; the two
// points of each half-vector are updated by packed FP32 pairs.  The 13
// coefficient vectors of a point are read from global memory at the point
// (the first 4 before the step's barrier, the rest at the start of the
// update): level 1 reads them for its halo'd tile, level 2 R + 1 steps later
// for the owned tile -- the second read is meant to hit L2 (all tiles of a
// plane march z together).  HBM then carries u^t, u^{t-1} and the 13 arrays
// once and the two written levels once per two time steps.
// Points outside the interior hold the zero Dirichlet value at level 1 (their
// value is selected to zero; their coefficients are not read).
// Level 2 and, for the next pass's u^{t-1}, level 1 are written for the owned
// points; the receiver trace of both levels as well.
//
// The constant wave (W25_CONST) runs the same pass with its 5 folded
// weights in registers and no coefficient arrays.  The adjoint of the
// 13-array kinds runs it with the transposed update (see the kernel).
//
// Measured (512^3, FP32, T = 64): 81 GLUP/s for W25_VAR and 86 for J25_VAR,
// against 103 and 112 for the one-level TMA sweep, so it is not the default;
// W25_CONST (T = 100) 190-194 against 438: one 4-point vector per warp and
// a barrier per step leave its short steps latency-bound; the adjoint of
// W25_VAR / J25_VAR 39 / 37 against 91 / 94 for the one-level adjoint.
// Earlier forms: one 256-thread CTA doing both levels in turn with all 13
// coefficient vectors prefetched (72 / 76 GLUP/s; 245 registers and 196 KB
// of rings leave 8 warps per SM, 28% issue activity); the same split by
// level with two planes in flight (60 GLUP/s for W25_VAR: its 213 KB of rings
// leave too little L1 for the coefficient loads in flight).
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
constexpr int NW1 = (NP1 + 31) / 32;           // level-1 warps (14)
constexpr int NW2 = NPO / 32;                  // level-2 warps (8)
constexpr int NT = 32 * (NW1 + NW2);           // threads (704)
// level-0 planes in flight: one for the 13-array kinds (a step there takes
// several microseconds, far longer than a plane's copy, and one plane keeps
// the wave kind's rings under the 196 KB shared-memory carve-out, leaving
// L1 room for the coefficient loads in flight); two for the constant wave,
// whose short steps would otherwise wait for every copy
constexpr int pd_of(int kind) { return kind == W25_CONST ? 2 : 1; }
// level 2 updates plane q - 2R - 1 in step q, one plane behind the level-1
// plane q - R written in the same step, so the two levels need no barrier
// between them: level 0 keeps planes q - 2R - 1 .. q + PD, level 1 planes
// q - 3R - 1 .. q - R
constexpr int ns0_of(int kind) { return 2 * R + 2 + pd_of(kind); }   // level-0 slots
constexpr int nsp_of(int kind) { return pd_of(kind) + 1; }           // u^{t-1} slots
constexpr int NS1 = 2 * R + 2;                 // level-1 slots (10)
constexpr int P0 = TX0 * TY0, P1 = TX1 * TY1;  // plane sizes (floats)
static_assert((P0 * 4) % 128 == 0 && (P1 * 4) % 128 == 0, "128-byte aligned planes");
static_assert(NPO % 32 == 0, "whole level-2 warps");
// coefficient vectors of a point loaded before the step's barrier (the
// rest at the start of its update): measured at 512^3, T = 64, W25_VAR /
// J25_VAR GLUP/s: 0 -> 76 / 81, 4 -> 81 / 86, 7 -> 82 / 72, 13 -> 50 / 54
// (the 80 registers a 704-thread CTA allows then spill)
constexpr int NPF = 4;
constexpr size_t smem_of(int kind) {
    const bool wave = kind != J25_VAR;
    return 4 * ((size_t)ns0_of(kind) * P0 + (wave ? (size_t)nsp_of(kind) * P1 : 0) + (size_t)NS1 * P1) +
           8 * ns0_of(kind) + 16 + 128;
}
}  // namespace b25

// ADJ: the adjoint pass of the 13-array kinds (lam^t = g^t + A^T lam^{t+1}
// [+ 2 lam^{t+1} - lam^{t+2} for the wave kind]; a.u = lam^{t+1}, a.u_prev =
// lam^{t+2}): the transposed update gathers every term's coefficient at its
// source point, (A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k) -- for the x terms
// three aligned vectors of the axis array around the point, for y and z
// the vectors of the rows and planes +-d -- read from global memory at
// use (L1 / L2 serve the overlap between neighbouring points).  The residual
// plane of level k (a.inject + (k-1) a.inject_step) is added on plane
// rcv_z at every computed interior point, the halo'd level-1 points
// included.  Both levels are written (out_prev = level 1, out = level 2).
template <int KIND, bool ADJ = false>
__global__ void __launch_bounds__(b25::NT, 1)
blk25_kernel(const BlockedArgs<float> a, const __grid_constant__ CUtensorMap tm_u,
             const __grid_constant__ CUtensorMap tm_p) {
    using namespace b25;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr bool CW = KIND == W25_CONST;   // constant weights: no coefficient arrays
    static_assert(!(ADJ && CW), "the constant wave is symmetric: its adjoint is the forward pass");
    constexpr int PD = pd_of(KIND), NS0 = ns0_of(KIND), NSP = nsp_of(KIND);
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *const s0 = reinterpret_cast<float *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    float *const sp = s0 + NS0 * P0;                      // u^{t-1} slots (wave kind)
    float *const s1 = sp + (WAVE ? NSP * P1 : 0);         // level-1 slots
    uint64_t *const bars = reinterpret_cast<uint64_t *>(s1 + NS1 * P1);
    volatile int &abort_word = *reinterpret_cast<volatile int *>(bars + NS0);

    const Geom &g = a.g;
    const int tid = threadIdx.x;
    const bool lev1 = tid < 32 * NW1;                      // warp role: level 1 or level 2
    const int xo = blockIdx.x * TXO + R, yo = blockIdx.y * TYO + R;   // padded origin of the owned tile
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int qs = z0 - 2 * R, qe = z1 + 2 * R;            // level-0 planes this chunk reads: [qs, qe)
    const int64_t sz = g.sz, sy = g.sy, nf = g.nfield;
    const int64_t plane_elems = (int64_t)g.nx * g.ny;

    // level-1 thread: vector k = tid of the level-1 tile (k < NP1)
    const int k1 = lev1 ? tid : 0;
    const bool act1 = lev1 && k1 < NP1;
    const int r1 = act1 ? k1 / NV1 : 0, c1 = act1 ? (k1 % NV1) * V : 0;
    const int py1 = yo - R + r1, px1 = xo - R + c1;
    const bool in1 = act1 && py1 >= R && py1 < g.ny + R && px1 >= R && px1 < g.nx + R;
    const int64_t g1 = in1 ? (int64_t)py1 * sy + px1 : 0;
    const bool own1 = in1 && r1 >= R && r1 < R + TYO && c1 >= R && c1 < R + TXO;
    // level-2 thread: owned vector k2
    const int k2 = lev1 ? 0 : tid - 32 * NW1;
    const int r2 = k2 / NVO, c2 = (k2 % NVO) * V;
    const int py2 = yo + r2, px2 = xo + c2;
    const bool in2 = !lev1 && py2 < g.ny + R && px2 < g.nx + R;
    const int64_t g2 = in2 ? (int64_t)py2 * sy + px2 : 0;

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
    // c of planes of width W in the ring at buf, whose 9 planes around the
    // centre (z offsets -R..R) start at the float offsets pl[0..8]; the 13
    // coefficient vectors are read at the point (cf: array 0) as they are
    // needed.  The two points of each half-vector are updated by packed
    // FP32 pairs (FADD2 / FMUL2 / FFMA2): the scalar form's terms in its
    // order.
    // cf: the first NPF coefficient vectors of the point, loaded before the
    // step's barrier; the rest are read from cfp (array 0 at the point) at
    // the start of the update, so that their latency overlaps the first
    // terms
    // constant wave: the folded weights s0 .. s4
    float sc[R + 1];
#pragma unroll
    for (int d = 0; d <= R; ++d) sc[d] = (float)a.s.c[d];
    (void)sc;
    auto update = [&](const float *buf, const uint32_t (&pl)[2 * R + 1], int W, int r, int c, const float4 (&cf)[NPF],
                      const float *cfp, float4 prev) -> float4 {
        float4 cl[NPF < 13 ? 13 - NPF : 1];
        if constexpr (!CW) {
#pragma unroll
            for (int t = NPF; t < 13; ++t) cl[t - NPF] = __ldg(reinterpret_cast<const float4 *>(cfp + t * nf));
        }
        auto coef = [&](int t) { return t < NPF ? cf[t] : cl[t - NPF]; };
        const int rc = r * W + c;
        const float *C = buf + pl[R] + rc;
        const float4 cv = *reinterpret_cast<const float4 *>(C);
        const float4 lv = *reinterpret_cast<const float4 *>(C - V);
        const float4 rv = *reinterpret_cast<const float4 *>(C + V);
        const float cc[4] = {cv.x, cv.y, cv.z, cv.w};
        const float ll[4] = {lv.x, lv.y, lv.z, lv.w};
        const float rr[4] = {rv.x, rv.y, rv.z, rv.w};
        if constexpr (CW) {
            // the constant wave (weights folded on the host: s0 = 2 + alpha w0,
            // s_d = alpha w_d): s0 u - u^{t-1} + sum_d s_d ((x pair + y pair) + z pair)
            const float2 s0 = make_float2(sc[0], sc[0]);
            float2 a0 = __ffma2_rn(s0, make_float2(cv.x, cv.y), make_float2(-prev.x, -prev.y));
            float2 a1 = __ffma2_rn(s0, make_float2(cv.z, cv.w), make_float2(-prev.z, -prev.w));
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                const float4 yu = *reinterpret_cast<const float4 *>(C - d * W);
                const float4 yd = *reinterpret_cast<const float4 *>(C + d * W);
                const float4 zd = *reinterpret_cast<const float4 *>(buf + pl[R - d] + rc);
                const float4 zu = *reinterpret_cast<const float4 *>(buf + pl[R + d] + rc);
                float xs[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const float xl = i - d >= 0 ? cc[i - d] : ll[i - d + 4];
                    const float xr = i + d < 4 ? cc[i + d] : rr[i + d - 4];
                    xs[i] = xl + xr;
                }
                const float2 sd = make_float2(sc[d], sc[d]);
                const float2 t0 = __fadd2_rn(__fadd2_rn(make_float2(xs[0], xs[1]), __fadd2_rn(make_float2(yu.x, yu.y), make_float2(yd.x, yd.y))),
                                             __fadd2_rn(make_float2(zd.x, zd.y), make_float2(zu.x, zu.y)));
                const float2 t1 = __fadd2_rn(__fadd2_rn(make_float2(xs[2], xs[3]), __fadd2_rn(make_float2(yu.z, yu.w), make_float2(yd.z, yd.w))),
                                             __fadd2_rn(make_float2(zd.z, zd.w), make_float2(zu.z, zu.w)));
                a0 = __ffma2_rn(sd, t0, a0);
                a1 = __ffma2_rn(sd, t1, a1);
            }
            return make_float4(a0.x, a0.y, a1.x, a1.y);
        }
        const float4 w0 = coef(0);
        float2 a0 = __fmul2_rn(make_float2(w0.x, w0.y), make_float2(cv.x, cv.y));
        float2 a1 = __fmul2_rn(make_float2(w0.z, w0.w), make_float2(cv.z, cv.w));
        if constexpr (WAVE) {
            a0 = __fadd2_rn(__ffma2_rn(make_float2(2.0f, 2.0f), make_float2(cv.x, cv.y), a0), make_float2(-prev.x, -prev.y));
            a1 = __fadd2_rn(__ffma2_rn(make_float2(2.0f, 2.0f), make_float2(cv.z, cv.w), a1), make_float2(-prev.z, -prev.w));
        }
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            const float4 wx = coef(3 * d - 2), wy = coef(3 * d - 1), wz = coef(3 * d);
            const float4 yu = *reinterpret_cast<const float4 *>(C - d * W);
            const float4 yd = *reinterpret_cast<const float4 *>(C + d * W);
            const float4 zd = *reinterpret_cast<const float4 *>(buf + pl[R - d] + rc);
            const float4 zu = *reinterpret_cast<const float4 *>(buf + pl[R + d] + rc);
            float xs[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float xl = i - d >= 0 ? cc[i - d] : ll[i - d + 4];
                const float xr = i + d < 4 ? cc[i + d] : rr[i + d - 4];
                xs[i] = xl + xr;
            }
            a0 = __ffma2_rn(make_float2(wx.x, wx.y), make_float2(xs[0], xs[1]), a0);
            a1 = __ffma2_rn(make_float2(wx.z, wx.w), make_float2(xs[2], xs[3]), a1);
            a0 = __ffma2_rn(make_float2(wy.x, wy.y), __fadd2_rn(make_float2(yu.x, yu.y), make_float2(yd.x, yd.y)), a0);
            a1 = __ffma2_rn(make_float2(wy.z, wy.w), __fadd2_rn(make_float2(yu.z, yu.w), make_float2(yd.z, yd.w)), a1);
            a0 = __ffma2_rn(make_float2(wz.x, wz.y), __fadd2_rn(make_float2(zd.x, zd.y), make_float2(zu.x, zu.y)), a0);
            a1 = __ffma2_rn(make_float2(wz.z, wz.w), __fadd2_rn(make_float2(zd.z, zd.w), make_float2(zu.z, zu.w)), a1);
        }
        return make_float4(a0.x, a0.y, a1.x, a1.y);
    };

    // transposed update (ADJ) at a 4-point vector: tile row r, column c of
    // the ring planes as in update; Wp = array 0 at the vector's first point
    auto update_adj = [&](const float *buf, const uint32_t (&pl)[2 * R + 1], int W, int r, int c, const float *Wp,
                          float4 prev) -> float4 {
        auto ld = [](const float *p) { return __ldg(reinterpret_cast<const float4 *>(p)); };
        auto el = [](const float4 &v, int i) { return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w; };
        const int rc = r * W + c;
        const float *C = buf + pl[R] + rc;
        const float4 cv = *reinterpret_cast<const float4 *>(C);
        const float4 lv = *reinterpret_cast<const float4 *>(C - V);
        const float4 rv = *reinterpret_cast<const float4 *>(C + V);
        const float4 w0 = ld(Wp);
        float acc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            acc[i] = el(w0, i) * el(cv, i);
            if constexpr (WAVE) acc[i] = fma(2.0f, el(cv, i), acc[i]) - el(prev, i);
        }
#pragma unroll
        for (int d = 1; d <= R; ++d) {
            const float *wx = Wp + (3 * d - 2) * nf, *wy = Wp + (3 * d - 1) * nf, *wz = Wp + (3 * d) * nf;
            const float4 xa = ld(wx - V), xb = ld(wx), xc = ld(wx + V);          // x axis array, columns c-4 .. c+7
            const float4 ya = ld(wy - d * sy), yb = ld(wy + d * sy);            // rows -d, +d
            const float4 za = ld(wz - d * sz), zb = ld(wz + d * sz);            // planes -d, +d
            const float4 yu = *reinterpret_cast<const float4 *>(C - d * W);
            const float4 yd = *reinterpret_cast<const float4 *>(C + d * W);
            const float4 zd = *reinterpret_cast<const float4 *>(buf + pl[R - d] + rc);
            const float4 zu = *reinterpret_cast<const float4 *>(buf + pl[R + d] + rc);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const float wl = i - d >= 0 ? el(xb, i - d) : el(xa, i - d + 4);
                const float ll_ = i - d >= 0 ? el(cv, i - d) : el(lv, i - d + 4);
                const float wr = i + d < 4 ? el(xb, i + d) : el(xc, i + d - 4);
                const float rr_ = i + d < 4 ? el(cv, i + d) : el(rv, i + d - 4);
                acc[i] = fma(wl, ll_, acc[i]);
                acc[i] = fma(wr, rr_, acc[i]);
                acc[i] = fma(el(ya, i), el(yu, i), acc[i]);
                acc[i] = fma(el(yb, i), el(yd, i), acc[i]);
                acc[i] = fma(el(za, i), el(zd, i), acc[i]);
                acc[i] = fma(el(zb, i), el(zu, i), acc[i]);
            }
        }
        return make_float4(acc[0], acc[1], acc[2], acc[3]);
    };
    (void)update_adj;
    // residual of level k on the receiver plane (adjoint), 4 interior points
    // of tile row py, column px (padded)
    auto inject = [&](float4 &v, int k, int py, int px) {
        const float *inj = a.inject + (k - 1) * a.inject_step + (int64_t)(py - R) * g.nx + (px - R);
        v.x += inj[0]; v.y += inj[1]; v.z += inj[2]; v.w += inj[3];
    };
    (void)inject;

    // ring slots, advanced by one per step (no division in the loop):
    // s_in = level-0 slot of plane q, s_p = u^{t-1} slot of plane q,
    // s1c = level-1 slot of plane q - R
    int s_in = 0, s_p = 0, s1c = NS1 - R;   // plane qs - R sits in level-1 slot (-R) mod NS1
    uint32_t par = 0;                        // phase of level-0 slot s_in's barrier
    bool stop = false;
    // steps qs .. qe: level 1 at plane q - R while level-0 plane q exists
    // (q < qe), level 2 at plane q - 2R - 1 (the last step has no level 1)
    for (int q = qs; q <= qe && !stop; ++q) {
        // the 13 coefficient vectors of this step's point (level 1: plane
        // q - R, level 2: plane q - 2R - 1), issued before the wait and the
        // barrier so that their latency overlaps them
        float4 cf[NPF];
        const int pc = lev1 ? q - R : q - 2 * R - 1;
        const float *const cfp = CW ? nullptr : a.W + ((int64_t)(pc + R) * sz + (lev1 ? g1 : g2));
        if constexpr (!CW && !ADJ) {
            const bool on = lev1 ? (in1 && q >= qs + 2 * R && q < qe && (unsigned)pc < (unsigned)g.nz)
                                 : (in2 && q >= qs + 4 * R + 1);
#pragma unroll
            for (int t = 0; t < NPF; ++t)
                cf[t] = on ? __ldg(reinterpret_cast<const float4 *>(cfp + t * nf)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (q < qe) bad |= !pv::mbar_wait_or_abort(&bars[s_in], par, wlim, &abort_word);
        if ((q - qs) % 8 == 7) stop = __syncthreads_or(bad);
        else __syncthreads();
        if (tid == 0 && q + PD < qe) issue(q + PD);
        if (lev1) {
            // ---- level 1 at plane pc1 (level-1 tile), into level-1 slot s1c
            const int pc1 = q - R;
            const bool l1on = q >= qs + 2 * R && q < qe;
            if (l1on && act1) {
                uint32_t pl0[2 * R + 1];   // level-0 planes pc1 - R .. pc1 + R = q - 2R .. q
#pragma unroll
                for (int i = 0; i <= 2 * R; ++i) {
                    int sl = s_in - 2 * R + i;
                    sl += sl < 0 ? NS0 : 0;
                    pl0[i] = (uint32_t)(sl * P0);
                }
                float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (WAVE) prev = *reinterpret_cast<const float4 *>(sp + s_p * P1 + r1 * TX1 + c1);
                float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
                if (in1 && (unsigned)pc1 < (unsigned)g.nz) {
                    if constexpr (ADJ) {
                        v = update_adj(s0, pl0, TX0, r1 + R, c1 + R, cfp, prev);
                        if (a.inject && pc1 == a.rcv_z) inject(v, 1, py1, px1);
                    } else {
                        v = update(s0, pl0, TX0, r1 + R, c1 + R, cf, cfp, prev);
                    }
                }
                *reinterpret_cast<float4 *>(s1 + s1c * P1 + r1 * TX1 + c1) = v;
                if (own1 && (unsigned)pc1 - (unsigned)z0 < (unsigned)(z1 - z0)) {
                    const int64_t o = (int64_t)(pc1 + R) * sz + g1;
                    if (a.out_prev && dbg_store_ok(a.dbg, g, o, V)) *reinterpret_cast<float4 *>(a.out_prev + o) = v;
                    if (a.trace && pc1 == a.rcv_z) {
                        float *tr = a.trace + (int64_t)(py1 - R) * g.nx + (px1 - R);
                        tr[0] = v.x; tr[1] = v.y; tr[2] = v.z; tr[3] = v.w;
                    }
                }
            }
        } else {
            // ---- level 2 at plane pc2 (owned tile): level-1 planes pc2-R..pc2+R
            const int pc2 = q - 2 * R - 1;
            if (q >= qs + 4 * R + 1 && in2) {
                uint32_t pl1[2 * R + 1];   // level-1 planes pc2 - R .. pc2 + R = q - 3R - 1 .. q - R - 1
#pragma unroll
                for (int i = 0; i <= 2 * R; ++i) {
                    int sl = s1c - 2 * R - 1 + i;
                    sl += sl < 0 ? NS1 : 0;
                    pl1[i] = (uint32_t)(sl * P1);
                }
                float4 prev = make_float4(0.f, 0.f, 0.f, 0.f);
                if constexpr (WAVE) {   // level 0 at plane pc2 = q - 2R - 1 (tile offset 2R)
                    int sl = s_in - 2 * R - 1;
                    sl += sl < 0 ? NS0 : 0;
                    prev = *reinterpret_cast<const float4 *>(s0 + sl * P0 + (r2 + 2 * R) * TX0 + c2 + 2 * R);
                }
                float4 v;
                if constexpr (ADJ) {
                    v = update_adj(s1, pl1, TX1, r2 + R, c2 + R, cfp, prev);
                    if (a.inject && pc2 == a.rcv_z) inject(v, 2, py2, px2);
                } else {
                    v = update(s1, pl1, TX1, r2 + R, c2 + R, cf, cfp, prev);
                }
                const int64_t o = (int64_t)(pc2 + R) * sz + g2;
                if (dbg_store_ok(a.dbg, g, o, V)) *reinterpret_cast<float4 *>(a.out + o) = v;
                if (a.trace && pc2 == a.rcv_z) {
                    float *tr = a.trace + plane_elems + (int64_t)(py2 - R) * g.nx + (px2 - R);
                    tr[0] = v.x; tr[1] = v.y; tr[2] = v.z; tr[3] = v.w;
                }
            }
        }
        // advance the ring slots
        if (++s_in == NS0) { s_in = 0; par ^= 1u; }
        if (++s_p == NSP) s_p = 0;
        if (++s1c == NS1) s1c = 0;
    }
    if (__syncthreads_or(bad) && tid == 0) {
        for (int qq = max(last_issued - PD + 1, qs); qq <= last_issued; ++qq)
            pv::mbar_wait(&bars[(qq - qs) % NS0], (uint32_t)(((qq - qs) / NS0) & 1), wlim);
        atomicAdd(&g_wait_timeouts, 1u);
    }
}

// Whether the two-level pass serves the plan: FP32, the 13-array kinds and
// the constant wave, 2 levels, whole 4-point vectors along x, planes below
// 2^30 points.
inline bool blk25_supported(int kind, int levels, const Geom &g) {
    return (kind == W25_VAR || kind == J25_VAR || kind == W25_CONST) && levels == 2 && g.nx % 4 == 0 &&
           (int64_t)g.px * g.py < ((int64_t)1 << 30);
}

// Resources (as stencil_pass_info reports them).
inline bool blk25_info(int kind, int64_t *info) {
    using namespace b25;
    if (kind != W25_VAR && kind != J25_VAR && kind != W25_CONST) return false;
    info[0] = (int64_t)smem_of(kind);
    info[1] = NT;
    info[2] = TX1;
    info[3] = TY1;
    info[4] = TXO;
    info[5] = TYO;
    return true;
}

inline cudaError_t launch_blk25(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms,
                                bool adjoint = false) {
    using namespace b25;
    const bool wave = kind != J25_VAR;   // W25_VAR, W25_CONST: second order in time
    CUtensorMap tm_u, tm_p;
    memset(&tm_u, 0, sizeof(tm_u));
    memset(&tm_p, 0, sizeof(tm_p));
    cudaError_t e = pv::make_tmap(&tm_u, a.u, 4, a.g, TX0, TY0);
    if (e == cudaSuccess && wave) e = pv::make_tmap(&tm_p, a.u_prev, 4, a.g, TX1, TY1);
    if (e != cudaSuccess) return e;
    const size_t smem = smem_of(kind);
    if (adjoint && kind == W25_CONST) return cudaErrorNotSupported;
    auto kern = adjoint ? (kind == W25_VAR ? blk25_kernel<W25_VAR, true> : blk25_kernel<J25_VAR, true>)
                        : (kind == W25_VAR ? blk25_kernel<W25_VAR> : kind == W25_CONST ? blk25_kernel<W25_CONST>
                                                                                        : blk25_kernel<J25_VAR>);
    static_assert(smem_of(W25_VAR) <= 227 * 1024 && smem_of(W25_CONST) <= 227 * 1024, "shared memory per CTA");
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
        const double cost = (double)((ctas + resident - 1) / resident) * (chunk + 4 * R + 1);
        if (cost < best_cost * 0.999) { best_cost = cost; best = nzc; }
    }
    BlockedArgs<float> b = a;
    b.zchunk = (a.g.nz + best - 1) / best;
    dim3 grid(gx, gy, (a.g.nz + b.zchunk - 1) / b.zchunk), block(NT, 1, 1);
    kern<<<grid, block, smem, st>>>(b, tm_u, tm_p);
    return cudaGetLastError();
}

}  // namespace stc
