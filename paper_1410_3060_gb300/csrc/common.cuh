// common.cuh -- shared device helpers and kernel argument structs of
// libstencil.so.  Operator kinds and the padded layout are those of
// include/stencil.h (paper Sect. 3.1, Fig. 1).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace stc {

enum Kind { J7_CONST = 1, J7_VAR = 2, W25_CONST = 3, W25_VAR = 4, J25_VAR = 5, W25_ALPHA = 6 };

template <int K> struct KindTraits;
template <> struct KindTraits<J7_CONST>  { static constexpr int R = 1, NARR = 0; static constexpr bool WAVE = false; };
template <> struct KindTraits<J7_VAR>    { static constexpr int R = 1, NARR = 7; static constexpr bool WAVE = false; };
template <> struct KindTraits<W25_CONST> { static constexpr int R = 4, NARR = 0; static constexpr bool WAVE = true; };
template <> struct KindTraits<W25_VAR>   { static constexpr int R = 4, NARR = 13; static constexpr bool WAVE = true; };
template <> struct KindTraits<J25_VAR>   { static constexpr int R = 4, NARR = 13; static constexpr bool WAVE = false; };
template <> struct KindTraits<W25_ALPHA> { static constexpr int R = 4, NARR = 1; static constexpr bool WAVE = true; };

inline int kind_radius(int kind) {
    switch (kind) {
    case J7_CONST: case J7_VAR: return 1;
    case W25_CONST: case W25_VAR: case J25_VAR: case W25_ALPHA: return 4;
    default: return -1;
    }
}
inline int kind_arrays(int kind) {
    switch (kind) {
    case J7_VAR: return 7;
    case W25_VAR: case J25_VAR: return 13;
    case W25_ALPHA: return 1;
    default: return 0;
    }
}
inline int kind_weights(int kind) {
    switch (kind) {
    case J7_CONST: return 2;
    case W25_CONST: return 6;
    case W25_ALPHA: return 5;
    default: return 0;
    }
}
inline bool kind_wave(int kind) { return kind == W25_CONST || kind == W25_VAR || kind == W25_ALPHA; }

// Padded geometry.  Extents fit in int (checked at plan time); strides and
// the field size are 64-bit.
struct Geom {
    int nx, ny, nz;      // interior
    int px, py, pz;      // padded = n + 2R
    int64_t sy, sz;      // strides in elements (sx = 1)
    int64_t nfield;      // px * py * pz
};

// Scalars folded on the host per kind (see plain.cu for their meaning).
struct Scalars { double c[6]; };

// Arguments of one plain sweep launch (one time level).
template <typename T>
struct SweepArgs {
    const T *u_prev;     // level t-1 (second-order kinds); may alias out
    const T *u;          // level t (stencil field)
    T *out;              // level t+1
    const T *W;          // coefficient stack [k][pz][py][px] (variable kinds)
    T *trace;            // trace plane [ny][nx] for this step, or nullptr
    const T *inject;     // adjoint: residual plane [ny][nx] added on rcv plane, or nullptr
    Scalars s;
    Geom g;
    int rcv_z;           // interior z of the receiver plane (trace / inject)
    int zchunk;          // interior planes per CTA along z
    int variant;         // forward tile variant (0 = default of the kind / dtype)
    int wait_limit;      // polls of a bounded mbarrier wait before it gives up (TMA-staged kernels)
    int skip_plane;      // test hook: the first CTA does not issue the copy of this plane (SKIP_NONE = off)
    unsigned long long *dbg;   // debug builds: first bad store index + 1 (nullptr otherwise)
};

// Polls of a bounded mbarrier wait when a plan sets no limit.
constexpr int WAIT_LIMIT_DEFAULT = 1 << 22;
// skip_plane value that matches no plane.
constexpr int SKIP_NONE = -(1 << 30);

// ---- cp.async (LDGSTS) helpers: 4- or 8-byte element copies into shared
// memory; any element-aligned global address works.
template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    if constexpr (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
    else if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
// cp.async that writes zeros instead of reading when `valid` is false (the
// source operand size is then 0 and nothing is read).
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill(void *smem, const void *gmem, bool valid) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    const int src = valid ? BYTES : 0;
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async sizes");
    if constexpr (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src) : "memory");
    else if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src) : "memory");
}
// cp.async of BYTES bytes that reads src_bytes (BYTES or 0) and zero-fills
// the rest; gmem must be a valid address either way.
template <int BYTES>
__device__ __forceinline__ void cp_async_zfill_n(void *smem, const void *gmem, uint32_t src_bytes) {
    const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16, "cp.async sizes");
    if constexpr (BYTES == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
    else if constexpr (BYTES == 8)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__host__ __device__ constexpr int cmod(int a, int m) { return ((a % m) + m) % m; }

// Debug build (-DSTENCIL_DEBUG): every store of a sweep's result checks that
// its n points, from linear index idx on, are interior points of the padded
// array (a sweep never writes the halo); a store that fails is skipped and
// its index recorded in *dbg (the first one wins).  It never traps.  In the
// normal build the check is the constant true.
#ifdef STENCIL_DEBUG
__device__ __forceinline__ bool dbg_store_ok(unsigned long long *dbg, const Geom &g, int64_t idx, int n = 1) {
    const int R = (g.px - g.nx) / 2;
    bool ok = idx >= 0 && idx + n <= g.nfield;
    if (ok) {
        const int64_t z = idx / g.sz, r = idx - z * g.sz, y = r / g.sy, x = r - y * g.sy;
        ok = z >= R && z < g.nz + R && y >= R && y < g.ny + R && x >= R && x + n - 1 < g.nx + R;
    }
    if (!ok && dbg) atomicCAS(dbg, 0ull, (unsigned long long)(idx + 1));
    return ok;
}
#else
__device__ __forceinline__ constexpr bool dbg_store_ok(unsigned long long *, const Geom &, int64_t, int = 1) {
    return true;
}
#endif

// Compile-time loop: f(IC<0>{}), ..., f(IC<N-1>{}); the index is a constant
// expression inside f (used for register-ring slots).
template <int V> struct IC { static constexpr int value = V; };
template <int N, int I = 0, typename F>
__device__ __forceinline__ void static_for(F &&f) {
    if constexpr (I < N) {
        f(IC<I>{});
        static_for<N, I + 1>(f);
    }
}

}  // namespace stc
