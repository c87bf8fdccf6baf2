// plainv_impl.cuh -- vectorised plain sweep (one level per launch) of the
// 25-point kinds (Fig. 1d, 1e structures, R = 4), written for few
// instructions per lattice update.
//
// Per thread: V consecutive x points (16-byte vectors: 4 FP32 or 2 FP64
// values) of one row; a warp covers 32 V columns, a CTA WY rows.  The field
// plane (tile plus an R-point halo on every side) is staged by cp.async PD
// planes ahead into a ring of shared slots (16-byte copies, zero fill outside
// the padded array); x and y neighbours are 16-byte shared loads (R is a
// multiple of V, so every neighbour vector is aligned); the 2R+1 planes along
// z of the thread's points live in a register ring (the step loop is unrolled
// by 2R+1 so ring slots are registers); u^{t-1} and the coefficients of the
// thread's points are 16-byte global loads.  Compared with the one-point-per-
// thread kernels every address, copy and load serves V points.
//
// TMA staging (template flag TMA): one thread issues each plane tile (and the
// per-point planes) as a single cp.async.bulk.tensor copy described by a
// tensor map, completing on a per-slot mbarrier that every thread waits on;
// the tensor unit zero-fills everything outside the padded array.  The copy
// then costs no per-thread instructions.  The wait is bounded: a thread
// whose wait runs out raises a shared abort word, and every other wait of
// the CTA that is still polling sees the word and gives up at once; the
// issuing thread stops issuing after its own wait failed (so no copy is ever
// issued into a slot whose copy may still be in flight).  Every thread still
// passes every barrier; the CTA agrees on leaving at the barrier of the last
// step of each unrolled block of planes and after the loop
// (__syncthreads_or -- one reduction barrier per 2R+1 planes: a reduction
// barrier after every plane cost 13% of the constant wave's speed), then the
// issuing thread waits (bounded again) for the copies it still has in
// flight, counts one timeout in a device counter and the CTA returns; its
// planes are wrong.  stencil_check turns the counter into STENCIL_ETIMEOUT.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <string.h>

#include "plain.cuh"

namespace stc {

namespace pv {

template <typename T> struct V16;
template <> struct V16<float> { using type = float4; static constexpr int n = 4; };
template <> struct V16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void ld16(T (&d)[V16<T>::n], const T *p) {
    const auto v = *reinterpret_cast<const typename V16<T>::type *>(p);
    if constexpr (V16<T>::n == 4) {
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    } else {
        d[0] = v.x; d[1] = v.y;
    }
}
template <typename T>
__device__ __forceinline__ void ldg16(T (&d)[V16<T>::n], const T *p) {
    const auto v = __ldg(reinterpret_cast<const typename V16<T>::type *>(p));
    if constexpr (V16<T>::n == 4) {
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    } else {
        d[0] = v.x; d[1] = v.y;
    }
}
template <typename T>
__device__ __forceinline__ void st16(T *p, const T (&s)[V16<T>::n]) {
    typename V16<T>::type v;
    if constexpr (V16<T>::n == 4) {
        v.x = s[0]; v.y = s[1]; v.z = s[2]; v.w = s[3];
    } else {
        v.x = s[0]; v.y = s[1];
    }
    *reinterpret_cast<typename V16<T>::type *>(p) = v;
}

template <typename T, int KIND, int WY, bool ADJ = false, bool TMA = false>
struct Tile {
    static constexpr int R = KindTraits<KIND>::R;
    static constexpr int V = V16<T>::n;
    static constexpr int TX = 32 * V, TY = WY;
    static constexpr int RH = (R + V - 1) / V * V;   // halo columns, whole vectors
    static constexpr int OS = R - R % V;             // own columns of tile bx start at bx TX + OS (aligned)
    static constexpr int SW = TX + 2 * RH, SH = TY + 2 * R, SP0 = SW * SH;
    static constexpr int SP = (int)((SP0 * sizeof(T) + 127) / 128 * 128 / sizeof(T));   // slot stride
    // per-point inputs staged with the field plane: u^{t-1} (second-order
    // kinds) and a single coefficient array (alpha); 13-array kinds load
    // their coefficients directly
    static constexpr int NPS = (KindTraits<KIND>::WAVE ? 1 : 0) + ((KindTraits<KIND>::NARR == 1 && !ADJ) ? 1 : 0);
    static constexpr int PP = TX * TY;           // one per-point plane
    static constexpr size_t smem_of(int pd) {
        // slots, per-point planes, one mbarrier per slot, the abort word
        // (16 bytes) and 128 bytes for the alignment of the first slot
        return sizeof(T) * ((size_t)(R + 1 + pd) * SP + (size_t)(R + 1 + pd) * NPS * PP) + 8 * (R + 1 + pd) + 16 + 128;
    }
    // planes in flight: one more with TMA (its copies take no registers) for
    // the constant wave (measured: 448 vs 402 GLUP/s at 512^3) and the
    // forward of the alpha-array wave, where the larger ring fits; the
    // 13-array kinds run slower with it
    static constexpr bool DEEP = TMA && !ADJ && KindTraits<KIND>::NARR <= 1 && KindTraits<KIND>::WAVE;
    static constexpr int PD = (DEEP && smem_of(3) <= 227 * 1024) ? 3 : 2;
    static constexpr int NS = R + 1 + PD;        // shared plane slots
    static constexpr size_t smem = smem_of(PD);
    static_assert((sizeof(T) * SP) % 128 == 0 && (sizeof(T) * PP) % 128 == 0, "128-byte aligned slots");
    static constexpr int MINB = 1;
};

// ---- TMA / mbarrier helpers (inline PTX)
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// 3D tile copy global -> shared, completing on `bar`; coordinates are
// elements (x innermost); x * element size must be a multiple of 16 bytes
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int x, int y, int z, uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(b), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for phase `parity` of `bar`; false when `limit` polls gave up
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, int limit) {
    const uint32_t b = smem_u32(bar);
    for (int it = 0; it < limit; ++it)
        if (mbar_try(b, parity)) return true;
    return false;
}
// the same, also giving up as soon as another thread of the CTA raised the
// shared abort word; a wait that runs out raises it
__device__ __forceinline__ bool mbar_wait_or_abort(uint64_t *bar, uint32_t parity, int limit, volatile int *abort_word) {
    const uint32_t b = smem_u32(bar);
    if (mbar_try(b, parity)) return true;
    for (int it = 1; it < limit; ++it) {
        if (mbar_try(b, parity)) return true;
        if ((it & 31) == 0 && *abort_word) return false;
    }
    *abort_word = 1;
    return false;
}

}  // namespace pv

// CTAs whose bounded wait gave up (a counter per translation unit; read
// through plainv_timeouts_f32 / _f64).
static __device__ unsigned int g_wait_timeouts;

namespace pv {
// Polls of a bounded wait for this launch.
__device__ __forceinline__ int wait_limit_of(int v) { return v > 0 ? v : WAIT_LIMIT_DEFAULT; }
// Test hook: whether this CTA skips issuing the copies of plane q.
__device__ __forceinline__ bool skip_copy(int skip_plane, int q) {
    return q == skip_plane && blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0;
}
}  // namespace pv

// ADJ: the adjoint (transposed) sweep of a variable-coefficient kind: every
// term's coefficient is read at its source point,
// (A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k); x-shifted coefficients come
// from the three (FP32) or five (FP64) aligned vectors around the own one.
template <typename T, int KIND, int WY, bool ADJ = false, bool TMA = false>
__global__ void __launch_bounds__(32 * WY, pv::Tile<T, KIND, WY, ADJ, TMA>::MINB)
plainv_kernel(const SweepArgs<T> a, const __grid_constant__ CUtensorMap tm_u,
              const __grid_constant__ CUtensorMap tm_p, const __grid_constant__ CUtensorMap tm_a) {
    using TL = pv::Tile<T, KIND, WY, ADJ, TMA>;
    constexpr int R = TL::R, V = TL::V;
    constexpr bool WAVE = KindTraits<KIND>::WAVE;
    constexpr int NA = KindTraits<KIND>::NARR;
    constexpr int RH = TL::RH, OS = TL::OS, SP0 = TL::SP0;
    constexpr int RING = 2 * R + 1;
    constexpr int PD = TL::PD, NS = TL::NS;
    constexpr int TX = TL::TX, TY = TL::TY, SW = TL::SW, SH = TL::SH, SP = TL::SP;
    static_assert(R % V == 0 || (R == 1 && KIND == J7_CONST) || (R == 1 && KIND == J7_VAR), "aligned own vectors");
    constexpr int VPR = SW / V;                  // vectors per shared row
    constexpr int NVEC = VPR * SH;               // vectors per plane
    constexpr int NT = 32 * WY;
    constexpr int NC = (NVEC + NT - 1) / NT;     // copies per thread per plane
    static_assert(NC <= 32, "copy mask");

    constexpr int NPS = TL::NPS, PP = TL::PP;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // slots start on 128-byte boundaries (TMA destinations); the launch adds
    // 128 bytes for this round-up
    T *const sb = reinterpret_cast<T *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
    T *const spp = sb + NS * SP;                 // [NS][NPS][TY][TX]
    uint64_t *const bars = reinterpret_cast<uint64_t *>(spp + NS * NPS * PP);   // TMA: one per slot
    (void)bars; (void)tm_u; (void)tm_p; (void)tm_a;

    const Geom &g = a.g;
    const int lane = threadIdx.x, w = threadIdx.y, tid = w * 32 + lane;
    const int xo = blockIdx.x * TX + OS;                      // padded column of the tile's first own point
    const int x0 = xo - RH, y0 = blockIdx.y * TY;            // padded origin of the shared tile
    const int z0 = blockIdx.z * a.zchunk;
    const int z1 = min(z0 + a.zchunk, g.nz);
    const int qs = z0 - R, qe = z1 + R;
    const int sy = (int)g.sy;
    const int64_t sz = g.sz;

    // copy plan: vector v = tid + c NT of the shared tile
    int goff[NC], soff[NC];
    uint32_t cmask = 0;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int v = tid + c * NT;
        const int row = v / VPR, vc = v - row * VPR;
        const int gx = x0 + vc * V, gy = y0 + row;
        goff[c] = gy * sy + gx;
        soff[c] = row * SW + vc * V;
        if (v < NVEC && gx >= 0 && gx < g.px && gy < g.py) cmask |= 1u << c;
        if (v >= NVEC) soff[c] = 0;
    }
    // this thread's points: padded row y0 + R + w, columns xo + lane V ..
    const int px = xo + lane * V, py = y0 + R + w;
    // radius 4 (nx % V == 0): a vector is wholly in or out of the interior;
    // radius 1: the vectors at the interior's x edges hold one halo point
    constexpr bool PARTIAL = (R % V) != 0;
    bool cin[V];
    bool call, own;   // own: any point of the vector is interior
    if constexpr (PARTIAL) {
        call = py < g.ny + R;
        own = false;
#pragma unroll
        for (int i = 0; i < V; ++i) {
            cin[i] = py < g.ny + R && px + i >= R && px + i < g.nx + R;
            call = call && cin[i];
            own = own || cin[i];
        }
    } else {
        own = px < g.nx + R && py < g.ny + R;
        call = own;
#pragma unroll
        for (int i = 0; i < V; ++i) cin[i] = own;
    }
    (void)call;
    const int poff = py * sy + px;
    const int scen = (R + w) * SW + RH + lane * V;     // shared offset of the own vector
    const int pown = w * TX + lane * V;                // offset in a per-point plane
    // bounded waits: whether a wait of this thread gave up; the issuing
    // thread's last issued plane (the copies possibly in flight when the CTA
    // leaves are among the last PD it issued)
    bool bad = false;
    int last_issued = qs - 1;
    volatile int &abort_word = *reinterpret_cast<volatile int *>(bars + NS);   // raised by a wait that ran out
    (void)bad; (void)last_issued; (void)abort_word;
    // field plane q (tile and halo) and the per-point inputs of output plane
    // q - R into slot `slot`
    auto issue = [&](int q, int slot) {
        if constexpr (TMA) {
            // thread 0: the tile with its halo, and the per-point planes of
            // output plane q - R (outside the padded array: zero fill)
            // the issuing thread stops after its own wait failed
            if (tid == 0 && !bad && !pv::skip_copy(a.skip_plane, q)) {
                last_issued = q;
                pv::mbar_expect_tx(&bars[slot], (uint32_t)(sizeof(T) * (SP0 + NPS * PP)));
                pv::tma_load_3d(sb + slot * SP, &tm_u, x0, y0, q + R, &bars[slot]);
                if constexpr (KindTraits<KIND>::WAVE)
                    pv::tma_load_3d(spp + slot * (NPS * PP), &tm_p, xo, y0 + R, q, &bars[slot]);
                if constexpr (NA == 1 && !ADJ)
                    pv::tma_load_3d(spp + slot * (NPS * PP) + (NPS - 1) * PP, &tm_a, xo, y0 + R, q, &bars[slot]);
            }
            return;
        }
        const bool zm = q >= -R && q < g.nz + R;
        const T *pb = a.u + (zm ? (int64_t)(q + R) * sz : 0);
        T *d = sb + slot * SP;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (tid + c * NT >= NVEC) continue;
            const bool ok = zm && ((cmask >> c) & 1u);
            cp_async_zfill<16>(d + soff[c], ok ? (const void *)(pb + goff[c]) : (const void *)a.u, ok);
        }
        if constexpr (NPS > 0) {
            // own points of planes this chunk computes only (an in-place
            // update overwrites u^{t-1} of the planes it owns)
            const int zq = q - R;
            const bool ok = own && zq >= z0 && zq < z1;
            const int64_t zo = ok ? (int64_t)(zq + R) * sz + poff : 0;
            T *dp = spp + slot * (NPS * PP) + pown;
            if constexpr (KindTraits<KIND>::WAVE)
                cp_async_zfill<16>(dp, ok ? (const void *)(a.u_prev + zo) : (const void *)a.u, ok);
            if constexpr (NA == 1 && !ADJ)
                cp_async_zfill<16>(dp + (NPS - 1) * PP, ok ? (const void *)(a.W + zo) : (const void *)a.u, ok);
        }
    };

    T ring[RING][V];
#pragma unroll
    for (int s = 0; s < RING; ++s)
#pragma unroll
        for (int i = 0; i < V; ++i) ring[s][i] = T(0);

    if constexpr (TMA) {
        if (tid < NS) pv::mbar_init(&bars[tid], 1);
        if (tid == 0) abort_word = 0;
        pv::mbar_init_fence();
        __syncthreads();
    }
#pragma unroll
    for (int s = 0; s < PD; ++s) {
        if (qs + s < qe) issue(qs + s, s);
        if constexpr (!TMA) cp_async_commit();
    }
    const T s0 = T(a.s.c[0]), s1 = T(a.s.c[1]), s2 = T(a.s.c[2]);
    const T s3 = T(a.s.c[3]), s4 = T(a.s.c[4]);
    (void)s0; (void)s1; (void)s2; (void)s3; (void)s4;

    int slot = 0;   // shared slot of plane q
    const int wlim = pv::wait_limit_of(a.wait_limit);
    (void)wlim;
    bool stop = false;   // CTA-uniform: a wait gave up (agreed at a reduction barrier)
    for (int qb = qs; qb < qe && !stop; qb += RING) {
        static_for<RING>([&](auto jj) {
            constexpr int j = decltype(jj)::value;
            const int q = qb + j;
            if (q >= qe) return;
            const int z = q - R;
            const int64_t zo = (int64_t)(z + R) * sz + poff;
            // 13-array kinds: the coefficients of output plane z, issued before
            // the wait so that their latency overlaps it
            T cf[NA > 1 ? NA : 1][V];
            (void)cf;
            if constexpr (NA > 1 && !ADJ) {
                if (own && z >= z0) {
#pragma unroll
                    for (int t = 0; t < NA; ++t) pv::ldg16<T>(cf[t], a.W + t * g.nfield + zo);
                } else {
#pragma unroll
                    for (int t = 0; t < NA; ++t)
#pragma unroll
                        for (int i = 0; i < V; ++i) cf[t][i] = T(0);
                }
            }
            if constexpr (TMA) {
                // k-th use of a slot completes phase k (parity k & 1)
                // (after a failure the abort word makes every later wait of
                // the block give up within a few polls)
                bad |= !pv::mbar_wait_or_abort(&bars[slot], (uint32_t)(((q - qs) / NS) & 1), wlim, &abort_word);
                // the CTA agrees on leaving once per unrolled block
                if constexpr (j == RING - 1) stop = __syncthreads_or(bad);
                else __syncthreads();
            } else {
                cp_async_wait<PD - 1>();
                __syncthreads();
            }
            pv::ld16<T>(ring[j], sb + slot * SP + scen);
            // staged per-point inputs of output plane z
            T pvv[V], al[V];
            (void)pvv; (void)al;
            if constexpr (KindTraits<KIND>::WAVE) pv::ld16<T>(pvv, spp + slot * (NPS * PP) + pown);
            if constexpr (NA == 1 && !ADJ) pv::ld16<T>(al, spp + slot * (NPS * PP) + (NPS - 1) * PP + pown);
            {
                int ns = slot + PD;
                if (ns >= NS) ns -= NS;
                if (q + PD < qe) issue(q + PD, ns);
                if constexpr (!TMA) cp_async_commit();
            }
            int zslot = slot - R;
            if (zslot < 0) zslot += NS;
            slot = slot + 1 == NS ? 0 : slot + 1;
            if (z < z0) return;
            // centre plane z: in-plane neighbours from shared memory
            const T *sc = sb + zslot * SP + scen;
            T lv[RH / V][V], rv[RH / V][V];   // the RH columns left and right of the own vector
#pragma unroll
            for (int m = 0; m < RH / V; ++m) {
                pv::ld16<T>(lv[m], sc - (m + 1) * V);   // columns -V(m+1) .. -V m - 1
                pv::ld16<T>(rv[m], sc + (m + 1) * V);   // columns V(m+1) .. V(m+2) - 1
            }
            T yv[2][R][V];
#pragma unroll
            for (int d = 1; d <= R; ++d) {
                pv::ld16<T>(yv[0][d - 1], sc - d * SW);
                pv::ld16<T>(yv[1][d - 1], sc + d * SW);
            }
            T res[V];
            // neighbour value of point i at x offset e (|e| <= R)
            auto xval = [&](int i, int e) -> T {
                const int c = i + e;   // column relative to the own vector start
                if (c < 0) {
                    const int m = (-c - 1) / V;            // vector m to the left
                    return lv[m][V - 1 - ((-c - 1) % V)];
                } else if (c >= V) {
                    const int m = (c - V) / V;
                    return rv[m][(c - V) % V];
                }
                return ring[cmod(j - R, RING)][c];
            };
            // adjoint: coefficient vector of array t at (dz planes, dy rows, dx
            // columns) from the own vector; dx a multiple of V
            auto cvec = [&](T (&d)[V], int t, int dz, int dy, int dx) {
                if (own) {
                    pv::ldg16<T>(d, a.W + t * g.nfield + zo + (int64_t)dz * sz + dy * sy + dx);
                } else {
#pragma unroll
                    for (int i = 0; i < V; ++i) d[i] = T(0);
                }
            };
            // x-shifted coefficients of array t: cl (R columns left), cm (own), cr (R right)
            auto cx_load = [&](int t, T (&cl)[RH / V][V], T (&cm)[V], T (&cr)[RH / V][V]) {
#pragma unroll
                for (int m = 0; m < RH / V; ++m) {
                    cvec(cl[m], t, 0, 0, -(m + 1) * V);
                    cvec(cr[m], t, 0, 0, (m + 1) * V);
                }
                cvec(cm, t, 0, 0, 0);
            };
            auto cx_at = [&](const T (&cl)[RH / V][V], const T (&cm)[V], const T (&cr)[RH / V][V], int c) -> T {
                if (c < 0) return cl[(-c - 1) / V][V - 1 - ((-c - 1) % V)];
                if (c >= V) return cr[(c - V) / V][(c - V) % V];
                return cm[c];
            };
            (void)cvec; (void)cx_load; (void)cx_at;
            if constexpr (ADJ && (KIND == W25_VAR || KIND == J25_VAR)) {
                T c0v[V];
                cvec(c0v, 0, 0, 0, 0);
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T c = ring[cmod(j - R, RING)][i];
                    res[i] = c0v[i] * c;
                    if constexpr (WAVE) res[i] = fma(T(2), c, res[i]) - pvv[i];
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int d = r + 1;
                    T cl[RH / V][V], cm[V], cr[RH / V][V], cyu[V], cyd[V], czd[V], czu[V];
                    cx_load(3 * r + 1, cl, cm, cr);
                    cvec(cyu, 3 * r + 2, 0, -d, 0);
                    cvec(cyd, 3 * r + 2, 0, d, 0);
                    cvec(czd, 3 * r + 3, -d, 0, 0);
                    cvec(czu, 3 * r + 3, d, 0, 0);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        T acc = res[i];
                        acc = fma(cx_at(cl, cm, cr, i - d), xval(i, -d), acc);
                        acc = fma(cx_at(cl, cm, cr, i + d), xval(i, d), acc);
                        acc = fma(cyu[i], yv[0][r][i], acc);
                        acc = fma(cyd[i], yv[1][r][i], acc);
                        acc = fma(czd[i], ring[cmod(j - R - d, RING)][i], acc);
                        acc = fma(czu[i], ring[cmod(j - R + d, RING)][i], acc);
                        res[i] = acc;
                    }
                }
            } else if constexpr (ADJ) {  // W25_ALPHA: A^T y = L (alpha y) + 2y - y_prev
                const T wr[4] = {s1, s2, s3, s4};
                T a0[V];
                cvec(a0, 0, 0, 0, 0);
                T sacc[V];
#pragma unroll
                for (int i = 0; i < V; ++i) sacc[i] = s0 * (a0[i] * ring[cmod(j - R, RING)][i]);
                T cl[RH / V][V], cr[RH / V][V];
                cx_load(0, cl, a0, cr);
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int d = r + 1;
                    T ayu[V], ayd[V], azd[V], azu[V];
                    cvec(ayu, 0, 0, -d, 0);
                    cvec(ayd, 0, 0, d, 0);
                    cvec(azd, 0, -d, 0, 0);
                    cvec(azu, 0, d, 0, 0);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        T pr = cx_at(cl, a0, cr, i - d) * xval(i, -d);
                        pr = fma(cx_at(cl, a0, cr, i + d), xval(i, d), pr);
                        pr = fma(ayu[i], yv[0][r][i], pr);
                        pr = fma(ayd[i], yv[1][r][i], pr);
                        pr = fma(azd[i], ring[cmod(j - R - d, RING)][i], pr);
                        pr = fma(azu[i], ring[cmod(j - R + d, RING)][i], pr);
                        sacc[i] = fma(wr[r], pr, sacc[i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T c = ring[cmod(j - R, RING)][i];
                    res[i] = sacc[i] + (T(2) * c - pvv[i]);
                }
            } else if constexpr (KIND == J7_CONST) {
                // Fig. 1b, the plain sweep's expression
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T c = ring[cmod(j - R, RING)][i];
                    res[i] = s0 * c + s1 * (((xval(i, -1) + xval(i, 1)) + (yv[0][0][i] + yv[1][0][i])) +
                                            (ring[cmod(j - R - 1, RING)][i] + ring[cmod(j - R + 1, RING)][i]));
                }
            } else if constexpr (KIND == J7_VAR) {
                // Fig. 1c, the plain sweep's order of terms
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    T v = cf[0][i] * ring[cmod(j - R, RING)][i];
                    v = fma(cf[1][i], xval(i, -1), v);
                    v = fma(cf[2][i], xval(i, 1), v);
                    v = fma(cf[3][i], yv[0][0][i], v);
                    v = fma(cf[4][i], yv[1][0][i], v);
                    v = fma(cf[5][i], ring[cmod(j - R - 1, RING)][i], v);
                    v = fma(cf[6][i], ring[cmod(j - R + 1, RING)][i], v);
                    res[i] = v;
                }
            } else if constexpr (KIND == W25_VAR || KIND == J25_VAR) {
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T c = ring[cmod(j - R, RING)][i];
                    T acc = cf[0][i] * c;
                    if constexpr (WAVE) acc = fma(T(2), c, acc) - pvv[i];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const int d = r + 1;
                        acc = fma(cf[3 * r + 1][i], xval(i, -d) + xval(i, d), acc);
                        acc = fma(cf[3 * r + 2][i], yv[0][r][i] + yv[1][r][i], acc);
                        acc = fma(cf[3 * r + 3][i], ring[cmod(j - R - d, RING)][i] + ring[cmod(j - R + d, RING)][i], acc);
                    }
                    res[i] = acc;
                }
            } else {
                const T wr[4] = {s1, s2, s3, s4};
#pragma unroll
                for (int i = 0; i < V; ++i) {
                    const T c = ring[cmod(j - R, RING)][i];
                    if constexpr (KIND == W25_CONST) {
                        T acc = s0 * c - pvv[i];
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int d = r + 1;
                            acc = fma(wr[r], ((xval(i, -d) + xval(i, d)) + (yv[0][r][i] + yv[1][r][i])) +
                                                 (ring[cmod(j - R - d, RING)][i] + ring[cmod(j - R + d, RING)][i]),
                                      acc);
                        }
                        res[i] = acc;
                    } else {  // W25_ALPHA
                        T sacc = s0 * c;
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            const int d = r + 1;
                            sacc = fma(wr[r], ((xval(i, -d) + xval(i, d)) + (yv[0][r][i] + yv[1][r][i])) +
                                                  (ring[cmod(j - R - d, RING)][i] + ring[cmod(j - R + d, RING)][i]),
                                       sacc);
                        }
                        res[i] = fma(al[i], sacc, T(2) * c - pvv[i]);
                    }
                }
            }
            if (own) {
                if (z == a.rcv_z) {
                    const int64_t pl = (int64_t)(py - R) * g.nx + (px - R);
#pragma unroll
                    for (int i = 0; i < V; ++i) {
                        if (!cin[i]) continue;
                        if (a.inject) res[i] += a.inject[pl + i];
                        if (a.trace) a.trace[pl + i] = res[i];
                    }
                }
                if constexpr (PARTIAL) {
                    if (call) {
                        if (dbg_store_ok(a.dbg, g, zo, V)) pv::st16<T>(a.out + zo, res);
                    } else {
                        // a vector that straddles the edge of the interior
#pragma unroll
                        for (int i = 0; i < V; ++i)
                            if (cin[i] && dbg_store_ok(a.dbg, g, zo + i)) a.out[zo + i] = res[i];
                    }
                } else if (dbg_store_ok(a.dbg, g, zo, V)) {
                    pv::st16<T>(a.out + zo, res);
                }
            }
        });
    }
    if constexpr (TMA) {
        // a partial last block ends without the block's reduction barrier
        if (__syncthreads_or(bad) && tid == 0) {
            // the last PD copies the issuing thread issued may still be in
            // flight: wait, bounded, for each (a completed one returns at
            // once) before the CTA's shared memory is released, then count
            // the timeout
            for (int qq = max(last_issued - PD + 1, qs); qq <= last_issued; ++qq)
                pv::mbar_wait(&bars[(qq - qs) % NS], (uint32_t)(((qq - qs) / NS) & 1), wlim);
            atomicAdd(&g_wait_timeouts, 1u);
        }
    } else {
        cp_async_wait<0>();
    }
}

// Whether the vectorised sweep serves this kind and geometry.
template <typename T>
inline bool plainv_supported(int kind, const Geom &g) {
    constexpr int V = pv::V16<T>::n;
    if ((int64_t)g.px * g.py >= ((int64_t)1 << 30)) return false;
    if (kind_radius(kind) == 4) return g.nx % V == 0;
    // 7-point kinds: FP64 vectors of two with an even padded row (16-byte rows)
    return sizeof(T) == 8 && (kind == J7_CONST || kind == J7_VAR) && g.px % V == 0;
}

namespace pv {
// Tensor map of one padded field (3D: x fastest) with a box of bx x by x 1
// elements; the tensor unit fills zeros outside the array.  The encoder is
// the driver's, looked up through the runtime (no link against the driver
// library).
// `arrays` > 1: that many padded fields stored one after another, mapped as
// one volume of arrays x pz planes.
inline cudaError_t make_tmap(CUtensorMap *m, const void *base, int elem_bytes, const Geom &g, int bx, int by,
                             int arrays = 1) {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void *f = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !f) return e != cudaSuccess ? e : cudaErrorNotSupported;
        fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
    }
    const cuuint64_t dims[3] = {(cuuint64_t)g.px, (cuuint64_t)g.py, (cuuint64_t)g.pz * (cuuint64_t)arrays};
    const cuuint64_t strides[2] = {(cuuint64_t)g.px * elem_bytes, (cuuint64_t)g.px * g.py * elem_bytes};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t es[3] = {1, 1, 1};
    const CUresult r = fn(m, elem_bytes == 4 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                          const_cast<void *>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// Interior planes per z chunk: minimise (waves of resident CTAs) x (planes
// per chunk including the 2R planes a chunk re-reads).
inline int pick_zchunk(int nz, int R, int64_t tiles, int64_t resident) {
    int best = 1;
    double best_cost = 1e300;
    for (int nzc = 1; nzc <= nz; ++nzc) {
        const int chunk = (nz + nzc - 1) / nzc;
        if (nzc > 1 && chunk < 4 * R) break;
        const int64_t ctas = tiles * ((nz + chunk - 1) / chunk);
        const double cost = (double)((ctas + resident - 1) / resident) * (chunk + 2 * R);
        if (cost < best_cost * 0.999) { best_cost = cost; best = nzc; }
    }
    return (nz + best - 1) / best;
}

// Interior planes per z chunk for an HBM-bound kernel: the fewest chunks
// (the least re-read of 2R planes per chunk) that still give 80% of the
// resident CTA slots a CTA.
inline int pick_zchunk_traffic(int nz, int R, int64_t tiles, int64_t resident) {
    int chunk = nz;
    for (int nzc = 1; nzc <= nz; ++nzc) {
        const int c = (nz + nzc - 1) / nzc;
        if (nzc > 1 && c < 4 * R) break;
        chunk = c;
        if (tiles * ((nz + c - 1) / c) * 5 >= resident * 4) break;
    }
    return chunk;
}
}  // namespace pv

template <typename T, int KIND, int WY, bool ADJ = false, bool TMA = false>
cudaError_t launch_plainv(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    using TL = pv::Tile<T, KIND, WY, ADJ, TMA>;
    constexpr int R = TL::R;
    auto kern = plainv_kernel<T, KIND, WY, ADJ, TMA>;
    CUtensorMap tm_u, tm_p, tm_a;
    memset(&tm_u, 0, sizeof(tm_u));
    memset(&tm_p, 0, sizeof(tm_p));
    memset(&tm_a, 0, sizeof(tm_a));
    if constexpr (TMA) {
        cudaError_t e = pv::make_tmap(&tm_u, a.u, sizeof(T), a.g, TL::SW, TL::SH);
        if (e == cudaSuccess && KindTraits<KIND>::WAVE) e = pv::make_tmap(&tm_p, a.u_prev, sizeof(T), a.g, TL::TX, TL::TY);
        if (e == cudaSuccess && KindTraits<KIND>::NARR == 1 && !ADJ) e = pv::make_tmap(&tm_a, a.W, sizeof(T), a.g, TL::TX, TL::TY);
        if (e != cudaSuccess) return e;
    }
    static_assert(TL::smem <= 227 * 1024, "shared memory per CTA");
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TL::smem);
    if (e != cudaSuccess) return e;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 32 * WY, TL::smem);
    if (per_sm < 1) per_sm = 1;
    const int gx = (a.g.nx + R - TL::OS + TL::TX - 1) / TL::TX, gy = (a.g.ny + TL::TY - 1) / TL::TY;
    SweepArgs<T> b = a;
    b.zchunk = pv::pick_zchunk(a.g.nz, R, (int64_t)gx * gy, (int64_t)num_sms * per_sm);
    dim3 grid(gx, gy, (a.g.nz + b.zchunk - 1) / b.zchunk), block(32, WY, 1);
    kern<<<grid, block, TL::smem, st>>>(b, tm_u, tm_p, tm_a);
    return cudaGetLastError();
}

}  // namespace stc

#include "adjt_impl.cuh"

namespace stc {

template <typename T, bool TMA>
cudaError_t launch_plainv_kind_t(int kind, bool adjoint, const SweepArgs<T> &a, bool big, cudaStream_t st,
                                 int num_sms) {
    if (adjoint) {  // variable kinds (the constant kind is self-adjoint: forward sweep below)
        // the 13-array adjoint runs 8-row tiles for both variants: its
        // source-point coefficients reach 4 rows up and down, which 8-row
        // tiles keep in L1 more often (measured: 142.7 vs 150.2 ms for the
        // 256^3 forward+adjoint backward pass)
        // with TMA staging the 13-array kinds run the staged-coefficient
        // adjoint (adjt_impl.cuh)
        switch (kind) {
        case W25_VAR: return TMA ? launch_adjt<T, W25_VAR, 8>(a, st, num_sms) : launch_plainv<T, W25_VAR, 8, true, false>(a, st, num_sms);
        case J25_VAR: return TMA ? launch_adjt<T, J25_VAR, 8>(a, st, num_sms) : launch_plainv<T, J25_VAR, 8, true, false>(a, st, num_sms);
        case W25_ALPHA: return big ? launch_plainv<T, W25_ALPHA, 4, true, TMA>(a, st, num_sms) : launch_plainv<T, W25_ALPHA, 8, true, TMA>(a, st, num_sms);
        case W25_CONST: break;
        default: return cudaErrorNotSupported;
        }
    }
    switch (kind) {
    case J7_CONST:
    case J7_VAR:
        if constexpr (sizeof(T) == 8) {   // FP64 7-point sweeps (FP32 rows of nx + 2 floats are not 16-byte aligned)
            if (kind == J7_CONST)
                return big ? launch_plainv<T, J7_CONST, 16, false, TMA>(a, st, num_sms) : launch_plainv<T, J7_CONST, 8, false, TMA>(a, st, num_sms);
            return big ? launch_plainv<T, J7_VAR, 16, false, TMA>(a, st, num_sms) : launch_plainv<T, J7_VAR, 8, false, TMA>(a, st, num_sms);
        }
        return cudaErrorNotSupported;
    case W25_CONST: return big ? launch_plainv<T, W25_CONST, 16, false, TMA>(a, st, num_sms) : launch_plainv<T, W25_CONST, 8, false, TMA>(a, st, num_sms);
    // the 13-array kinds hold 13 coefficient vectors per thread: their second
    // tile is 4 rows (more CTAs per SM) instead of 16
    case W25_VAR: return big ? launch_plainv<T, W25_VAR, 4, false, TMA>(a, st, num_sms) : launch_plainv<T, W25_VAR, 8, false, TMA>(a, st, num_sms);
    case J25_VAR: return big ? launch_plainv<T, J25_VAR, 4, false, TMA>(a, st, num_sms) : launch_plainv<T, J25_VAR, 8, false, TMA>(a, st, num_sms);
    case W25_ALPHA: return big ? launch_plainv<T, W25_ALPHA, 16, false, TMA>(a, st, num_sms) : launch_plainv<T, W25_ALPHA, 8, false, TMA>(a, st, num_sms);
    default: return cudaErrorNotSupported;
    }
}

// Variants 13 / 14: cp.async staging; 15 / 16: the same tiles with TMA staging.
template <typename T>
cudaError_t launch_plainv_kind(int kind, bool adjoint, const SweepArgs<T> &a, int variant, cudaStream_t st,
                               int num_sms) {
    const bool big = variant == 14 || variant == 16;
    if (variant >= 15) return launch_plainv_kind_t<T, true>(kind, adjoint, a, big, st, num_sms);
    return launch_plainv_kind_t<T, false>(kind, adjoint, a, big, st, num_sms);
}

// Resources of a forward configuration (as launch_plainv_kind selects it):
// dynamic shared memory, threads, tile extents (computed = owned).
template <typename T, int KIND, int WY, bool TMA>
bool plainv_info_cfg(int64_t *info) {
    using TL = pv::Tile<T, KIND, WY, false, TMA>;
    info[0] = (int64_t)TL::smem;
    info[1] = 32 * WY;
    info[2] = info[4] = TL::TX;
    info[3] = info[5] = TL::TY;
    return true;
}
template <typename T, bool TMA>
bool plainv_info_t(int kind, bool big, int64_t *info) {
    switch (kind) {
    case J7_CONST:
        if constexpr (sizeof(T) == 8) return big ? plainv_info_cfg<T, J7_CONST, 16, TMA>(info) : plainv_info_cfg<T, J7_CONST, 8, TMA>(info);
        return false;
    case J7_VAR:
        if constexpr (sizeof(T) == 8) return big ? plainv_info_cfg<T, J7_VAR, 16, TMA>(info) : plainv_info_cfg<T, J7_VAR, 8, TMA>(info);
        return false;
    case W25_CONST: return big ? plainv_info_cfg<T, W25_CONST, 16, TMA>(info) : plainv_info_cfg<T, W25_CONST, 8, TMA>(info);
    case W25_VAR: return big ? plainv_info_cfg<T, W25_VAR, 4, TMA>(info) : plainv_info_cfg<T, W25_VAR, 8, TMA>(info);
    case J25_VAR: return big ? plainv_info_cfg<T, J25_VAR, 4, TMA>(info) : plainv_info_cfg<T, J25_VAR, 8, TMA>(info);
    case W25_ALPHA: return big ? plainv_info_cfg<T, W25_ALPHA, 16, TMA>(info) : plainv_info_cfg<T, W25_ALPHA, 8, TMA>(info);
    default: return false;
    }
}
template <typename T>
bool plainv_info(int kind, int variant, int64_t *info) {
    if (variant < 13 || variant > 16) return false;
    const bool big = variant == 14 || variant == 16;
    return variant >= 15 ? plainv_info_t<T, true>(kind, big, info) : plainv_info_t<T, false>(kind, big, info);
}

// Waits of this translation unit's kernels that gave up.
inline unsigned int plainv_read_timeouts() {
    unsigned int v = 0;
    if (cudaMemcpyFromSymbol(&v, g_wait_timeouts, sizeof(v)) != cudaSuccess) return 0;
    return v;
}

}  // namespace stc
