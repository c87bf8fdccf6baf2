// aux.cu -- coefficient-gradient accumulation and the receiver misfit.
//
// Gradient (adjoint of the coefficient dependence of the update, for the
// variable-coefficient kinds): for every interior point x and every step n
// of a batch, grad_k(x) += lam^{n+1}(x) * d(A u^n)(x)/dA_k(x), where the
// derivative is the field value multiplying A_k in the update:
//   J7_VAR  (Fig. 1c): u^n(x + o_k), o_k in {0, -x, +x, -y, +y, -z, +z}
//   W25_VAR / J25_VAR (Fig. 1d structure): u^n(x) for k = 0, the pair
//           u^n(x + r e_a) + u^n(x - r e_a) for k = 3(r-1)+a+1
//   W25_ALPHA (Fig. 1e): w0 u^n(x) + sum_r w_r (pairs along x, y, z)
// The batch sum is added to the FP64 gradient arrays once per batch (see
// grad_kernel for how FP32 plans form it).
#include <algorithm>
#include <mutex>

#include "plain.cuh"

namespace stc {

// Per-step gradient terms d_k of one point (FP64 plans: in FP64; FP32
// plans: products of the FP32 fields formed in FP32).
template <typename T, int KIND>
__device__ __forceinline__ void grad_terms(const T *u, const T l, const Geom &g, const Scalars &s, T *d) {
    if constexpr (KIND == J7_VAR) {
        const int64_t o[7] = {0, -1, 1, -g.sy, g.sy, -g.sz, g.sz};
#pragma unroll
        for (int k = 0; k < 7; ++k) d[k] = l * u[o[k]];
    } else if constexpr (KIND == W25_VAR || KIND == J25_VAR) {
        d[0] = l * u[0];
        const int64_t st[3] = {1, g.sy, g.sz};
#pragma unroll
        for (int r = 1; r <= 4; ++r)
#pragma unroll
            for (int ax = 0; ax < 3; ++ax) {
                const int64_t off = r * st[ax];
                d[3 * (r - 1) + ax + 1] = l * (u[-off] + u[off]);
            }
    } else {  // W25_ALPHA: d(alpha L u)/d alpha = L u
        T sum = T(s.c[0]) * u[0];
#pragma unroll
        for (int r = 1; r <= 4; ++r) {
            const int64_t sy = g.sy, sz = g.sz;
            const T pr = ((u[-r] + u[r]) + (u[-r * sy] + u[r * sy])) + (u[-r * sz] + u[r * sz]);
            sum = fma(T(s.c[r]), pr, sum);
        }
        d[0] = l * sum;
    }
}

// One thread per interior point; loops over the batch of steps.  FP64
// plans accumulate the terms in FP64.  FP32 plans form each term in FP32
// (the fields are FP32) and sum the terms of the batch with compensated
// (Kahan) FP32 summation -- error of a few FP32 roundings of the batch sum,
// the order of the rounding of the FP32 terms themselves -- then add the
// batch sum, rounded once to FP32 (sum - compensation: one more rounding of
// the batch sum), to the FP64 gradient: the sum over time is carried in
// FP64.  GB300 runs FP64 at 2 operations per clock per SM, so the epilogue
// takes one conversion and one FP64 add per array.
template <typename T, int KIND>
__global__ void __launch_bounds__(256) grad_kernel(const GradArgs<T> a) {
    constexpr int R = KindTraits<KIND>::R;
    constexpr int NA = KindTraits<KIND>::NARR;
    const Geom g = a.g;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * 8 + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= g.nx || y >= g.ny) return;
    const int64_t idx = (int64_t)(z + R) * g.sz + (int64_t)(y + R) * g.sy + (x + R);
    // software pipeline: the terms of step s + 1 are loaded and formed before
    // the terms of step s are summed, so the loads of two steps are in flight
    T d[NA], dn[NA];
    if (a.nsteps > 0) grad_terms<T, KIND>(a.u[0] + idx, a.lam[0][idx], g, a.s, d);
    if constexpr (sizeof(T) == 8) {
        double acc[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) acc[k] = 0.0;
        for (int s = 0; s < a.nsteps; ++s) {
            if (s + 1 < a.nsteps) grad_terms<T, KIND>(a.u[s + 1] + idx, a.lam[s + 1][idx], g, a.s, dn);
#pragma unroll
            for (int k = 0; k < NA; ++k) acc[k] += d[k];
#pragma unroll
            for (int k = 0; k < NA; ++k) d[k] = dn[k];
        }
#pragma unroll
        for (int k = 0; k < NA; ++k) a.grad[(int64_t)k * g.nfield + idx] += acc[k];
    } else {
        float sum[NA], cmp[NA];
#pragma unroll
        for (int k = 0; k < NA; ++k) { sum[k] = 0.f; cmp[k] = 0.f; }
        for (int s = 0; s < a.nsteps; ++s) {
            if (s + 1 < a.nsteps) grad_terms<T, KIND>(a.u[s + 1] + idx, a.lam[s + 1][idx], g, a.s, dn);
#pragma unroll
            for (int k = 0; k < NA; ++k) {
                // compensated summation; __fadd_rn / __fsub_rn keep the
                // compensation from being reassociated away
                const float yk = __fsub_rn(d[k], cmp[k]);
                const float tk = __fadd_rn(sum[k], yk);
                cmp[k] = __fsub_rn(__fsub_rn(tk, sum[k]), yk);
                sum[k] = tk;
            }
#pragma unroll
            for (int k = 0; k < NA; ++k) d[k] = dn[k];
        }
#pragma unroll
        for (int k = 0; k < NA; ++k)
            a.grad[(int64_t)k * g.nfield + idx] += (double)__fsub_rn(sum[k], cmp[k]);
    }
}

// 25-point variable kinds, one axis per thread: the three threads of a
// point (threadIdx.z = axis a) sum the four radii of their axis, and the
// x-axis thread also the centre term.  The terms and the order of each sum
// are those of grad_kernel (the results are identical); a thread holds 5
// sums instead of 13, so that an SM keeps about three times as many warps,
// and loads, in flight.
template <typename T, int TY>
__global__ void __launch_bounds__(96 * TY, TY == 8 ? 2 : 3) grad_axis_kernel(const GradArgs<T> a) {
    constexpr int R = 4;
    const Geom g = a.g;
    const int x = blockIdx.x * 32 + threadIdx.x;
    const int y = blockIdx.y * TY + threadIdx.y;
    const int z = blockIdx.z;
    const int ax = threadIdx.z;            // warp-uniform
    if (x >= g.nx || y >= g.ny) return;
    const int64_t idx = (int64_t)(z + R) * g.sz + (int64_t)(y + R) * g.sy + (x + R);
    const int64_t st = ax == 0 ? 1 : (ax == 1 ? g.sy : g.sz);
    const bool centre = ax == 0;
    // d[r - 1]: radius r of this axis; d[4]: the centre term (axis 0)
    auto terms = [&](int s, T (&d)[5]) {
        const T *u = a.u[s] + idx;
        const T l = a.lam[s][idx];
#pragma unroll
        for (int r = 1; r <= 4; ++r) d[r - 1] = l * (u[-r * st] + u[r * st]);
        d[4] = centre ? l * u[0] : T(0);
    };
    T d[5], dn[5];
    if (a.nsteps > 0) terms(0, d);
    double out[5];
    if constexpr (sizeof(T) == 8) {
        double acc[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] = 0.0;
        for (int s = 0; s < a.nsteps; ++s) {
            if (s + 1 < a.nsteps) terms(s + 1, dn);
#pragma unroll
            for (int k = 0; k < 5; ++k) acc[k] += d[k];
#pragma unroll
            for (int k = 0; k < 5; ++k) d[k] = dn[k];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k] = acc[k];
    } else {
        float sum[5], cmp[5];
#pragma unroll
        for (int k = 0; k < 5; ++k) { sum[k] = 0.f; cmp[k] = 0.f; }
        for (int s = 0; s < a.nsteps; ++s) {
            if (s + 1 < a.nsteps) terms(s + 1, dn);
#pragma unroll
            for (int k = 0; k < 5; ++k) {
                const float yk = __fsub_rn(d[k], cmp[k]);
                const float tk = __fadd_rn(sum[k], yk);
                cmp[k] = __fsub_rn(__fsub_rn(tk, sum[k]), yk);
                sum[k] = tk;
            }
#pragma unroll
            for (int k = 0; k < 5; ++k) d[k] = dn[k];
        }
#pragma unroll
        for (int k = 0; k < 5; ++k) out[k] = (double)__fsub_rn(sum[k], cmp[k]);
    }
#pragma unroll
    for (int r = 1; r <= 4; ++r) a.grad[(int64_t)(3 * (r - 1) + ax + 1) * g.nfield + idx] += out[r - 1];
    if (centre) a.grad[idx] += out[4];
}

// 25-point variable kinds, tiles staged in shared memory.  Per step of the
// batch a CTA (one plane, GT_X x GT_Y points, one thread per point) copies
// with 16-byte cp.async chunks: the tile of u^n on its plane with x and y
// halos of R, the tile's own columns of u^n on the 2R planes z +- 1..R, and
// lam^{n+1} on the tile; the copies of the next NSLOT - 1 steps are in
// flight while a step is summed from shared memory.  The terms and the
// order of every sum are those of grad_kernel (identical results).  Needs
// 16-byte aligned rows: nx a multiple of 16 / sizeof(T).
constexpr int GT_X = 32, GT_Y = 8;
template <typename T>
struct GradTile {
    static constexpr int R = 4;
    static constexpr int VE = 16 / (int)sizeof(T);            // elements per chunk
    static constexpr int HW = GT_X + 2 * R, HH = GT_Y + 2 * R;  // halo tile
    static constexpr int HALO = HW * HH, ZB = 2 * R * GT_X * GT_Y, LAM = GT_X * GT_Y;
    static constexpr int SLOT = HALO + ZB + LAM;
    static constexpr int NCH = (HALO + ZB + LAM) / VE;         // chunks per step
    static constexpr int NT = GT_X * GT_Y;
    static constexpr int NC = (NCH + NT - 1) / NT;             // chunks per thread
    static constexpr int NSLOT = sizeof(T) == 4 ? 4 : 3;
    static constexpr size_t smem = sizeof(T) * (size_t)NSLOT * SLOT;
    static_assert(HW % VE == 0 && GT_X % VE == 0, "whole chunks per row");
};

template <typename T>
__global__ void __launch_bounds__(GT_X * GT_Y) grad_tile_kernel(const GradArgs<T> a) {
    using TL = GradTile<T>;
    constexpr int R = TL::R, VE = TL::VE, HW = TL::HW, NC = TL::NC, NSLOT = TL::NSLOT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *const sb = reinterpret_cast<T *>(smem_raw);
    const Geom g = a.g;
    const int lx = threadIdx.x, ly = threadIdx.y, tid = ly * GT_X + lx;
    const int x0 = blockIdx.x * GT_X, y0 = blockIdx.y * GT_Y;   // padded origin of the halo tile
    const int z = blockIdx.z;
    const int64_t zc = (int64_t)(z + R) * g.sz;
    // copy plan: chunk c = tid + i NT of a step; offsets relative to the
    // field base; `lm`: the chunk is lam's, else u's
    int soff[NC];
    int64_t goff[NC];
    uint32_t ok = 0, lm = 0, live = 0;
#pragma unroll
    for (int i = 0; i < NC; ++i) {
        int c = tid + i * TL::NT;
        soff[i] = 0;
        goff[i] = 0;
        if (c >= TL::NCH) continue;
        live |= 1u << i;
        int gx, gy;
        int64_t gz;
        if (c < TL::HALO / VE) {                        // halo tile of the plane
            const int row = c / (HW / VE), col = c % (HW / VE);
            soff[i] = row * HW + col * VE;
            gx = x0 + col * VE; gy = y0 + row; gz = zc;
        } else if ((c -= TL::HALO / VE) < TL::ZB / VE) {   // own columns, planes z -+ 1..R
            const int pl = c / (TL::LAM / VE), rem = c % (TL::LAM / VE);
            const int row = rem / (GT_X / VE), col = rem % (GT_X / VE);
            const int dz = pl < R ? -(pl + 1) : pl - R + 1;
            soff[i] = TL::HALO + pl * TL::LAM + row * GT_X + col * VE;
            gx = x0 + R + col * VE; gy = y0 + R + row; gz = zc + (int64_t)dz * g.sz;
        } else {                                        // lam on the tile
            c -= TL::ZB / VE;
            const int row = c / (GT_X / VE), col = c % (GT_X / VE);
            soff[i] = TL::HALO + TL::ZB + row * GT_X + col * VE;
            gx = x0 + R + col * VE; gy = y0 + R + row; gz = zc;
            lm |= 1u << i;
        }
        goff[i] = gz + (int64_t)gy * g.sy + gx;
        if (gx < g.px && gy < g.py) ok |= 1u << i;
    }
    auto issue = [&](int s) {
        T *d = sb + (s % NSLOT) * TL::SLOT;
        const T *u = a.u[s], *l = a.lam[s];
#pragma unroll
        for (int i = 0; i < NC; ++i) {
            if (!((live >> i) & 1u)) continue;
            const bool v = (ok >> i) & 1u;
            const T *src = ((lm >> i) & 1u) ? l : u;
            cp_async_zfill<16>(d + soff[i], v ? (const void *)(src + goff[i]) : (const void *)src, v);
        }
    };
    const bool in = x0 + lx < g.nx && y0 + ly < g.ny;
    const int hc = (ly + R) * HW + lx + R;             // own point in the halo tile
    const int oc = ly * GT_X + lx;                     // own point in a per-point tile
#pragma unroll
    for (int s = 0; s < NSLOT - 1; ++s) {
        if (s < a.nsteps) issue(s);
        cp_async_commit();
    }
    T d[13];
    float sum[13], cmp[13];
    double acc[13];
#pragma unroll
    for (int k = 0; k < 13; ++k) { sum[k] = 0.f; cmp[k] = 0.f; acc[k] = 0.0; }
    for (int s = 0; s < a.nsteps; ++s) {
        if (s + NSLOT - 1 < a.nsteps) issue(s + NSLOT - 1);   // into the slot of step s - 1
        cp_async_commit();
        cp_async_wait<NSLOT - 1>();
        __syncthreads();
        if (in) {
            const T *sl = sb + (s % NSLOT) * TL::SLOT;
            const T *h = sl + hc;
            const T l = sl[TL::HALO + TL::ZB + oc];
            d[0] = l * h[0];
#pragma unroll
            for (int r = 1; r <= 4; ++r) {
                d[3 * (r - 1) + 1] = l * (h[-r] + h[r]);
                d[3 * (r - 1) + 2] = l * (h[-r * HW] + h[r * HW]);
                d[3 * (r - 1) + 3] = l * (sl[TL::HALO + (r - 1) * TL::LAM + oc] + sl[TL::HALO + (R + r - 1) * TL::LAM + oc]);
            }
            if constexpr (sizeof(T) == 8) {
#pragma unroll
                for (int k = 0; k < 13; ++k) acc[k] += d[k];
            } else {
#pragma unroll
                for (int k = 0; k < 13; ++k) {
                    const float yk = __fsub_rn(d[k], cmp[k]);
                    const float tk = __fadd_rn(sum[k], yk);
                    cmp[k] = __fsub_rn(__fsub_rn(tk, sum[k]), yk);
                    sum[k] = tk;
                }
            }
        }
        __syncthreads();   // the slot of step s is refilled at step s + 1
    }
    cp_async_wait<0>();
    if (!in) return;
    const int64_t idx = zc + (int64_t)(y0 + R + ly) * g.sy + (x0 + R + lx);
#pragma unroll
    for (int k = 0; k < 13; ++k)
        a.grad[(int64_t)k * g.nfield + idx] += sizeof(T) == 8 ? acc[k] : (double)__fsub_rn(sum[k], cmp[k]);
}

template <typename T>
cudaError_t launch_grad(int kind, const GradArgs<T> &a, cudaStream_t st) {
    // batches of 8 or more steps: the staged tiles (256^3 FP32 under ncu, 16
    // steps: 2.66 against 3.13 ms); shorter batches, where the FP64
    // read-modify-write dominates: one thread per point and axis (4 steps:
    // 1.64 against 2.0 ms)
    if ((kind == W25_VAR || kind == J25_VAR) && a.g.nx % GradTile<T>::VE == 0 && a.nsteps >= 8) {
        using TL = GradTile<T>;
        cudaError_t e = cudaFuncSetAttribute(grad_tile_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)TL::smem);
        if (e != cudaSuccess) return e;
        dim3 block(GT_X, GT_Y, 1), grid((a.g.nx + GT_X - 1) / GT_X, (a.g.ny + GT_Y - 1) / GT_Y, a.g.nz);
        grad_tile_kernel<T><<<grid, block, TL::smem, st>>>(a);
        return cudaGetLastError();
    }
    if (kind == W25_VAR || kind == J25_VAR) {
        // FP32: 8 rows per CTA (the y neighbours of more rows stay in the
        // CTA); FP64: 4 rows (its 56 registers a thread allow three CTAs)
        constexpr int TY = sizeof(T) == 4 ? 8 : 4;
        dim3 block(32, TY, 3), grid((a.g.nx + 31) / 32, (a.g.ny + TY - 1) / TY, a.g.nz);
        grad_axis_kernel<T, TY><<<grid, block, 0, st>>>(a);
        return cudaGetLastError();
    }
    dim3 block(32, 8, 1), grid((a.g.nx + 31) / 32, (a.g.ny + 7) / 8, a.g.nz);
    switch (kind) {
    case J7_VAR: grad_kernel<T, J7_VAR><<<grid, block, 0, st>>>(a); break;
    case W25_ALPHA: grad_kernel<T, W25_ALPHA><<<grid, block, 0, st>>>(a); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// ---- misfit: residual = trace - d, partial sums of residual^2 per block in
// a grid-stride order that depends only on n, then one block sums the
// partials in index order.
template <typename T>
__global__ void __launch_bounds__(256) misfit_partial_kernel(const T *trace, const T *d, T *res, int64_t n,
                                                             double *partials) {
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const T r = trace[i] - d[i];
        res[i] = r;
        s = fma((double)r, (double)r, s);
    }
    __shared__ double sh[256];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void __launch_bounds__(256) misfit_final_kernel(const double *partials, int np, double *loss) {
    __shared__ double sh[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < np; i += 256) s += partials[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *loss = 0.5 * sh[0];
}

template <typename T>
cudaError_t launch_misfit(const T *trace, const T *d, T *residual, int64_t n, double *partials, int npartials,
                          double *loss, cudaStream_t st) {
    misfit_partial_kernel<T><<<npartials, 256, 0, st>>>(trace, d, residual, n, partials);
    misfit_final_kernel<<<1, 256, 0, st>>>(partials, npartials, loss);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(256) axpby_kernel(double alpha, const T *x, double beta, const T *y, T *out,
                                                    int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (T)(alpha * (double)x[i] + beta * (double)y[i]);
}

template <typename T>
cudaError_t launch_axpby(double alpha, const T *x, double beta, const T *y, T *out, int64_t n, int num_sms,
                         cudaStream_t st) {
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)num_sms * 16);
    axpby_kernel<T><<<(int)std::max<int64_t>(blocks, 1), 256, 0, st>>>(alpha, x, beta, y, out, n);
    return cudaGetLastError();
}

template cudaError_t launch_axpby<float>(double, const float *, double, const float *, float *, int64_t, int,
                                         cudaStream_t);
template cudaError_t launch_axpby<double>(double, const double *, double, const double *, double *, int64_t, int,
                                          cudaStream_t);
// ---- allocation-free misfit: the partial sums live in a library-owned
// static device array instead of plan scratch.  The array's name is only a
// host-side stand-in; its device address is looked up with the device
// current.  A call outside stream capture looks it up again (so the address
// stays right after a device reset reloads the module); a call inside a
// capture uses the address cached by an earlier call on that device and
// fails if there is none.
static __device__ __align__(256) double g_misfit_partials[MISFIT_STATIC_MAX_PARTIALS];

namespace {
std::mutex g_static_mtx;
constexpr int kMaxDevices = 64;
double *g_static_addr[kMaxDevices] = {};
}  // namespace

cudaError_t misfit_static(int dtype, const void *trace, const void *d, int64_t n, void *residual, double *loss,
                          cudaStream_t st) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess) return e;
    double *partials = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mtx);
        if (cap == cudaStreamCaptureStatusNone) {
            void *ptr = nullptr;
            e = cudaGetSymbolAddress(&ptr, g_misfit_partials);
            if (e != cudaSuccess) return e;
            g_static_addr[dev] = static_cast<double *>(ptr);
        } else if (!g_static_addr[dev]) {
            return cudaErrorStreamCaptureUnsupported;
        }
        partials = g_static_addr[dev];
    }
    // one partial sum per MISFIT_STATIC_ELEMS_PER_PARTIAL elements; every
    // partial the final sum reads is written by this call, so nothing has
    // to be cleared between calls
    const int np = (int)std::max<int64_t>(1, (n + MISFIT_STATIC_ELEMS_PER_PARTIAL - 1) / MISFIT_STATIC_ELEMS_PER_PARTIAL);
    if (dtype == 0)
        return launch_misfit<double>((const double *)trace, (const double *)d, (double *)residual, n, partials, np,
                                     loss, st);
    return launch_misfit<float>((const float *)trace, (const float *)d, (float *)residual, n, partials, np, loss,
                                st);
}

template cudaError_t launch_grad<float>(int, const GradArgs<float> &, cudaStream_t);
template cudaError_t launch_grad<double>(int, const GradArgs<double> &, cudaStream_t);
template cudaError_t launch_misfit<float>(const float *, const float *, float *, int64_t, double *, int, double *,
                                          cudaStream_t);
template cudaError_t launch_misfit<double>(const double *, const double *, double *, int64_t, double *, int,
                                           double *, cudaStream_t);

}  // namespace stc
