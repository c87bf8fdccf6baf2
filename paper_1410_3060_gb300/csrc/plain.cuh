// plain.cuh -- launchers of the kernels in plain.cu, aux.cu and blocked.cu.
#pragma once
#include "common.cuh"

namespace stc {

// Default forward tile variant of a kind and dtype (0 = FP64, 1 = FP32).
int default_variant(int kind, int dtype);

// One plain sweep (one time level), forward or adjoint.
template <typename T>
cudaError_t launch_plain(int kind, bool adjoint, const SweepArgs<T> &a, cudaStream_t st, int num_sms);

// Coefficient-gradient accumulation for `nsteps` adjoint steps:
// grad_k(x) += sum_s lam[s](x) * d(A u[s])(x)/dA_k(x) (FP64 accumulators).
constexpr int GRAD_MAX_STEPS = 16;
template <typename T>
struct GradArgs {
    const T *u[GRAD_MAX_STEPS];     // u^n of each step (padded)
    const T *lam[GRAD_MAX_STEPS];   // lam^{n+1} of each step (padded)
    double *grad;                   // [k][pz][py][px]
    Scalars s;                      // W25_ALPHA weights w0..w4
    Geom g;
    int nsteps;
};
template <typename T>
cudaError_t launch_grad(int kind, const GradArgs<T> &a, cudaStream_t st);

// residual = trace - d and loss = 0.5 sum residual^2 (FP64, fixed order).
template <typename T>
cudaError_t launch_misfit(const T *trace, const T *d, T *residual, int64_t n, double *partials,
                          int npartials, double *loss, cudaStream_t st);

// Misfit with its partial sums in a static device array (no allocation).
constexpr int MISFIT_STATIC_MAX_PARTIALS = 8192;          // 64 KiB of FP64
constexpr int64_t MISFIT_STATIC_ELEMS_PER_PARTIAL = 2048;
constexpr int64_t MISFIT_STATIC_MAX_ELEMS = (int64_t)MISFIT_STATIC_MAX_PARTIALS * MISFIT_STATIC_ELEMS_PER_PARTIAL;
cudaError_t misfit_static(int dtype, const void *trace, const void *d, int64_t n, void *residual, double *loss,
                          cudaStream_t st);

// out = alpha x + beta y over n elements
template <typename T>
cudaError_t launch_axpby(double alpha, const T *x, double beta, const T *y, T *out, int64_t n, int num_sms,
                         cudaStream_t st);

// Vectorised plain sweep of the 25-point kinds (plainv_impl.cuh): tile
// variant 13 = 8 rows per CTA, 14 = 16 rows per CTA (4 for the 13-array
// kinds); 15 and 16 the same tiles staged by TMA.  Served when the kind
// has radius 4 and nx is a multiple of the vector width (4 FP32, 2 FP64).
bool plainv_supported_f32(int kind, const Geom &g);
bool plainv_supported_f64(int kind, const Geom &g);
// bounded waits of the TMA-staged sweeps that gave up (device counters)
unsigned int plainv_timeouts_f32();
unsigned int plainv_timeouts_f64();
// resources of a forward variant 13-16 (see wavefront_info_f32)
bool plainv_info_f32(int kind, int variant, int64_t *info);
bool plainv_info_f64(int kind, int variant, int64_t *info);
template <typename T>
cudaError_t launch_plainv_kind(int kind, bool adjoint, const SweepArgs<T> &a, int variant, cudaStream_t st,
                               int num_sms);

// FP64 / FP32 FMA throughput probe.
cudaError_t run_fma_peak(int dtype, cudaStream_t st, double *flops, double *clock_hz);

}  // namespace stc
