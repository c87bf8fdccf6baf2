// adjt_impl.cuh -- adjoint (transposed) sweep of the 13-array 25-point kinds
// (Fig. 1d structure) with every operand staged by TMA; one level per launch.
// Included by plainv_impl.cuh (16-byte vector helpers, TMA / mbarrier
// helpers, tensor maps, the wait-timeout counter).
//
// The adjoint of u'(p) = sum_k A_k(p) u(p + o_k) reads every coefficient at
// the source point: (A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k).  A gather from
// global memory at the source points issues 29 dependent-latency vector
// loads per output vector after the plane wait.  Here each arriving plane p
// brings, into one shared slot and by one thread's bulk tensor copies:
//   the y tile of plane p with its x and y halos,
//   the 4 x-axis coefficient tiles of plane p with x halos (own rows),
//   the 4 y-axis coefficient tiles of plane p with y halos (own columns);
// the inputs of the thread's own points -- the centre and the 4 z-axis
// coefficients of plane p and y_prev (second-order kind) -- are 16-byte
// loads into registers issued while the thread waits for plane p.
// Every term of output plane p that reads plane p only -- the centre, the x
// and y terms, 2 y(p) - y_prev(p) -- is summed when plane p arrives.  The z
// terms are pushed: A_{z,r}(p) y(p) is added to the partial sums of output
// planes p - r and p + r (a register ring of 2R+1 partial sums), so output
// plane p - R is complete once plane p has arrived.  Three slots: the copies
// of planes p + 1 and p + 2 run while plane p is summed.  The plane waits are
// bounded and give up as in the forward sweep: a wait that runs out raises
// the CTA's abort word, the issuing thread stops issuing after its own wait
// failed, the CTA agrees on leaving once per unrolled block of planes and
// after the loop, and the issuing thread waits (bounded) for its copies in
// flight and counts one timeout.
#pragma once

namespace stc {

namespace pv {

template <typename T, int WY>
struct AdjTile {
    static constexpr int R = 4;
    static constexpr int V = V16<T>::n;
    static constexpr int TX = 32 * V, TY = WY;
    static constexpr int RH = (R + V - 1) / V * V;   // halo columns, whole vectors
    static constexpr int OS = R - R % V;             // own columns of tile bx start at bx TX + OS
    static constexpr int SW = TX + 2 * RH, SH = TY + 2 * R;
    // region sizes rounded to 128 bytes (TMA destinations)
    static constexpr int al(int n) { return (int)((n * sizeof(T) + 127) / 128 * 128 / sizeof(T)); }
    static constexpr int CXS = al(SW * TY), CYS = al(TX * SH);
    // element offsets of the regions of a slot
    static constexpr int LAM = 0;                    // [SH][SW]
    static constexpr int CX = LAM + al(SW * SH);     // 4 x [TY][SW]
    static constexpr int CY = CX + 4 * CXS;          // 4 x [SH][TX]
    static constexpr int SLOT = CY + 4 * CYS;
    static constexpr int NSLOT = 3;
    // bytes one plane's copies deliver (the boxes, zero fill included)
    static constexpr uint32_t BYTES = (uint32_t)sizeof(T) * (SW * SH + 4 * SW * TY + 4 * TX * SH);
    // slots, one mbarrier per slot, the abort word (16 bytes) and 128 bytes
    // for the alignment of the first slot
    static constexpr size_t smem = sizeof(T) * (size_t)NSLOT * SLOT + 8 * NSLOT + 16 + 128;
    static_assert((sizeof(T) * SLOT) % 128 == 0, "128-byte aligned slots");
};

}  // namespace pv

template <typename T, int KIND, int WY>
__global__ void __launch_bounds__(32 * WY, 1)
adjt_kernel(const SweepArgs<T> a, const __grid_constant__ CUtensorMap tm_lam, const __grid_constant__ CUtensorMap tm_cx,
            const __grid_constant__ CUtensorMap tm_cy) {
    using TL = pv::AdjTile<T, WY>;
    constexpr int R = TL::R, V = TL::V, TX = TL::TX, SW = TL::SW, RH = TL::RH, OS = TL::OS;
    constexpr int NH = RH / V;                   // halo vectors on each side
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int RING = 2 * R + 1;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *const sb = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    uint64_t *const bars = reinterpret_cast<uint64_t *>(sb + TL::NSLOT * TL::SLOT);

    const Geom &g = a.g;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
    const int xo = blockIdx.x * TX + OS, x0 = xo - RH, y0 = blockIdx.y * TL::TY;
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int qs = z0 - R, qe = z1 + R;
    const int pz = (int)g.pz;
    // this thread's points: padded row y0 + R + w, columns px .. px + V - 1
    // (nx is a multiple of V: a vector is wholly interior or wholly not)
    const int px = xo + lane * V, py = y0 + R + w;
    const bool own = px < g.nx + R && py < g.ny + R;
    const int64_t poff = (int64_t)py * g.sy + px;
    const int olam = (R + w) * SW + RH + lane * V;   // own vector in the y tile
    const int ocx = w * SW + RH + lane * V;          // ... in an x-axis tile
    const int ocy = (R + w) * TX + lane * V;         // ... in a y-axis tile

    // bounded waits: whether a wait of this thread gave up; the issuing
    // thread's last issued plane (the copies possibly in flight when the CTA
    // leaves are among the last two it issued)
    bool bad = false;
    int last_issued = qs - 1;
    volatile int &abort_word = *reinterpret_cast<volatile int *>(bars + TL::NSLOT);
    // all copies of plane p (interior index) into slot s (issuing thread)
    auto issue = [&](int p, int s) {
        if (bad || pv::skip_copy(a.skip_plane, p)) return;   // stopped, or the test hook's missing copy
        last_issued = p;
        T *d = sb + s * TL::SLOT;
        uint64_t *bar = &bars[s];
        const int zp = p + R;   // padded plane
        pv::mbar_expect_tx(bar, TL::BYTES);
        pv::tma_load_3d(d + TL::LAM, &tm_lam, x0, y0, zp, bar);
#pragma unroll
        for (int r = 1; r <= 4; ++r) {
            // array 3(r-1)+1: x axis, 3(r-1)+2: y axis
            pv::tma_load_3d(d + TL::CX + (r - 1) * TL::CXS, &tm_cx, x0, y0 + R, (3 * r - 2) * pz + zp, bar);
            pv::tma_load_3d(d + TL::CY + (r - 1) * TL::CYS, &tm_cy, xo, y0, (3 * r - 1) * pz + zp, bar);
        }
    };
    // own-point inputs of plane p: z-axis coefficients (array 3r) where p is
    // interior, the centre coefficient and y_prev where p is an output plane
    // of this chunk (y_prev may be the output array: only the chunk's own
    // planes are read, each before it is written)
    T pc0[V], pcz[4][V], plp[V];
    auto load_own = [&](int p) {
        const bool inz = own && p >= 0 && p < g.nz;
        const bool inc = own && p >= z0 && p < z1;
        const int64_t zo = (int64_t)(p + R) * g.sz + poff;
#pragma unroll
        for (int r = 1; r <= 4; ++r) {
            if (inz) {
                pv::ldg16<T>(pcz[r - 1], a.W + 3 * r * g.nfield + zo);
            } else {
#pragma unroll
                for (int i = 0; i < V; ++i) pcz[r - 1][i] = T(0);
            }
        }
        if (inc) {
            pv::ldg16<T>(pc0, a.W + zo);
            if constexpr (WAVE) pv::ld16<T>(plp, a.u_prev + zo);
        } else {
#pragma unroll
            for (int i = 0; i < V; ++i) pc0[i] = plp[i] = T(0);
        }
    };

    T acc[RING][V];   // partial sums of output planes p - R .. p + R (slot of plane p: its ring index)
#pragma unroll
    for (int s = 0; s < RING; ++s)
#pragma unroll
        for (int i = 0; i < V; ++i) acc[s][i] = T(0);

    if (tid < TL::NSLOT) pv::mbar_init(&bars[tid], 1);
    if (tid == 0) abort_word = 0;
    pv::mbar_init_fence();
    __syncthreads();
    if (tid == 0) {
        issue(qs, 0);
        if (qs + 1 < qe) issue(qs + 1, 1);
    }
    load_own(qs);
    static_assert(RING % TL::NSLOT == 0, "slot of plane p: j mod NSLOT");

    const int wlim = pv::wait_limit_of(a.wait_limit);
    bool stop = false;   // CTA-uniform: a wait gave up (agreed at a reduction barrier)
    for (int pb = qs; pb < qe && !stop; pb += RING) {
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            constexpr int s = j % TL::NSLOT;
            const int p = pb + j;
            if (p >= qe) return;
            // k-th use of a slot completes phase k (parity k & 1)
            bad |= !pv::mbar_wait_or_abort(&bars[s], (uint32_t)(((p - qs) / TL::NSLOT) & 1), wlim, &abort_word);
            // the barrier makes every thread done with plane p - 1's slot; the
            // CTA agrees on leaving once per unrolled block
            if constexpr (j == RING - 1) stop = __syncthreads_or(bad);
            else __syncthreads();
            if (tid == 0 && p + 2 < qe) issue(p + 2, (j + 2) % TL::NSLOT);
            const T *sl = sb + s * TL::SLOT;
            if (own && p >= 0 && p < g.nz) {
                T lc[V];
                pv::ld16<T>(lc, sl + TL::LAM + olam);
                // z terms with source plane p
#pragma unroll
                for (int r = 1; r <= 4; ++r) {
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        const T v = pcz[r - 1][i] * lc[i];
                        acc[cmod(j - r, RING)][i] += v;
                        acc[cmod(j + r, RING)][i] += v;
                    }
                }
                if (p >= z0 && p < z1) {
                    // terms of output plane p that read plane p only
                    T t[V];
#pragma unroll
                    for (int i = 0; i < V; ++i) t[i] = pc0[i] * lc[i];
                    if constexpr (WAVE) {
#pragma unroll
                        for (int i = 0; i < V; ++i) t[i] = fma(T(2), lc[i], t[i]) - plp[i];
                    }
                    // y vectors left and right of the own one (RH columns each side)
                    T ll[NH][V], lr[NH][V];
#pragma unroll
                    for (int m = 0; m < NH; ++m) {
                        pv::ld16<T>(ll[m], sl + TL::LAM + olam - (m + 1) * V);
                        pv::ld16<T>(lr[m], sl + TL::LAM + olam + (m + 1) * V);
                    }
                    // value at column c relative to the own vector start (|c| <= R + V - 1)
                    auto at = [&](const T (&l)[NH][V], const T (&o)[V], const T (&rr)[NH][V], int c) -> T {
                        if (c < 0) return l[(-c - 1) / V][V - 1 - ((-c - 1) % V)];
                        if (c >= V) return rr[(c - V) / V][(c - V) % V];
                        return o[c];
                    };
#pragma unroll
                    for (int r = 1; r <= 4; ++r) {
                        const T *cxr = sl + TL::CX + (r - 1) * TL::CXS + ocx;
                        T cl[NH][V], cm[V], cr[NH][V];
#pragma unroll
                        for (int m = 0; m < NH; ++m) {
                            pv::ld16<T>(cl[m], cxr - (m + 1) * V);
                            pv::ld16<T>(cr[m], cxr + (m + 1) * V);
                        }
                        pv::ld16<T>(cm, cxr);
                        const T *cyr = sl + TL::CY + (r - 1) * TL::CYS + ocy;
                        T cyu[V], cyd[V], lyu[V], lyd[V];
                        pv::ld16<T>(cyu, cyr - r * TX);
                        pv::ld16<T>(cyd, cyr + r * TX);
                        pv::ld16<T>(lyu, sl + TL::LAM + olam - r * SW);
                        pv::ld16<T>(lyd, sl + TL::LAM + olam + r * SW);
#pragma unroll
                        for (int i = 0; i < V; ++i) {
                            T v = t[i];
                            v = fma(at(cl, cm, cr, i - r), at(ll, lc, lr, i - r), v);
                            v = fma(at(cl, cm, cr, i + r), at(ll, lc, lr, i + r), v);
                            v = fma(cyu[i], lyu[i], v);
                            v = fma(cyd[i], lyd[i], v);
                            t[i] = v;
                        }
                    }
#pragma unroll
                    for (int i = 0; i < V; ++i) acc[j][i] += t[i];
                }
            }
            // output plane z = p - R is complete
            const int z = p - R;
            constexpr int jz = cmod(j - R, RING);
            if (own && z >= z0 && z < z1) {
                T res[V];
#pragma unroll
                for (int i = 0; i < V; ++i) res[i] = acc[jz][i];
                if (z == a.rcv_z) {
                    const int64_t pl = (int64_t)(py - R) * g.nx + (px - R);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        if (a.inject) res[i] += a.inject[pl + i];
                        if (a.trace) a.trace[pl + i] = res[i];
                    }
                }
                const int64_t zo = (int64_t)(z + R) * g.sz + poff;
                if (dbg_store_ok(a.dbg, g, zo, V)) pv::st16<T>(a.out + zo, res);
            }
#pragma unroll
            for (int i = 0; i < V; ++i) acc[jz][i] = T(0);   // now the slot of plane p + R + 1
            if (p + 1 < qe) load_own(p + 1);
        });
    }
    // a partial last block ends without the block's reduction barrier
    if (__syncthreads_or(bad) && tid == 0) {
        // the last two copies issued may still be in flight: wait, bounded,
        // for each (a completed one returns at once), then count the timeout
        for (int pp = max(last_issued - 1, qs); pp <= last_issued; ++pp)
            pv::mbar_wait(&bars[(pp - qs) % TL::NSLOT], (uint32_t)(((pp - qs) / TL::NSLOT) & 1), wlim);
        atomicAdd(&g_wait_timeouts, 1u);
    }
}

template <typename T, int KIND, int WY>
cudaError_t launch_adjt(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    using TL = pv::AdjTile<T, WY>;
    constexpr int R = TL::R, NA = KindTraits<KIND>::NARR;
    static_assert(NA == 13, "13-array kinds");
    auto kern = adjt_kernel<T, KIND, WY>;
    CUtensorMap m_lam, m_cx, m_cy;
    memset(&m_lam, 0, sizeof(m_lam));
    memset(&m_cx, 0, sizeof(m_cx));
    memset(&m_cy, 0, sizeof(m_cy));
    cudaError_t e = pv::make_tmap(&m_lam, a.u, sizeof(T), a.g, TL::SW, TL::SH);
    if (e == cudaSuccess) e = pv::make_tmap(&m_cx, a.W, sizeof(T), a.g, TL::SW, TL::TY, NA);
    if (e == cudaSuccess) e = pv::make_tmap(&m_cy, a.W, sizeof(T), a.g, TL::TX, TL::SH, NA);
    if (e != cudaSuccess) return e;
    static_assert(TL::smem <= 227 * 1024, "shared memory per CTA");
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WY, TL::smem);
    if (per_sm < 1) per_sm = 1;
    const int gx = (a.g.nx + R - TL::OS + TL::TX - 1) / TL::TX, gy = (a.g.ny + TL::TY - 1) / TL::TY;
    SweepArgs<T> b = a;
    // FP32: HBM-bound, the fewest chunks when they fit in one wave of
    // resident CTAs (measured at 256^3: 2 chunks of 128 planes, 121.8 ms for
    // the backward pass against 123.7 with the 7 chunks of the wave-count
    // choice); otherwise, and for FP64 (bound by the FP64 pipe), the
    // wave-count choice: a partial last wave of one-CTA-per-SM tiles costs
    // more than the re-read it saves
    const int64_t tiles = (int64_t)gx * gy, resident = (int64_t)num_sms * per_sm;
    b.zchunk = pv::pick_zchunk(a.g.nz, R, tiles, resident);
    if (sizeof(T) == 4) {
        const int c = pv::pick_zchunk_traffic(a.g.nz, R, tiles, resident);
        if (tiles * ((a.g.nz + c - 1) / c) <= resident) b.zchunk = c;
    }
    dim3 grid(gx, gy, (a.g.nz + b.zchunk - 1) / b.zchunk), block(32, WY, 1);
    kern<<<grid, block, TL::smem, st>>>(b, m_lam, m_cx, m_cy);
    return cudaGetLastError();
}

}  // namespace stc
