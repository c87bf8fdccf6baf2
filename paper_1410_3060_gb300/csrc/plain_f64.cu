// plain_f64.cu -- double instantiations of the plain sweeps (plain_impl.cuh).
#include "plain_impl.cuh"

namespace stc {

// Tile variants of the streaming forward kernel (TX threads in x, BY thread
// rows, NR rows per thread, PD planes of prefetch), selected per plan
// (STENCIL_OPT_VARIANT): 1 = 32x8x1/2, 2 = 32x8x2/2, 3 = 32x4x4/2,
// 4 = 64x4x2/2, 5 = the register-staged plain kernel (plain_sweep_kernel),
// 6 = 64x4x4/2, 7 = 128x2x4/2; 8 = 32x8x1/3 and 9 = 32x8x2/2 with the
// per-point inputs (coefficients, u^{t-1}) also staged by cp.async.
// 0 picks the default of the kind and dtype (measured best).
template <typename T, int KIND>
static cudaError_t launch_forward(const SweepArgs<T> &a, cudaStream_t st, int num_sms, int variant) {
    constexpr int R = KindTraits<KIND>::R;
    if (variant == 0) variant = default_variant(KIND, sizeof(T) == 8 ? 0 : 1);
    switch (variant) {
    case 1: return launch_stream<T, KIND, 32, 8, 1, 2>(a, st, num_sms);
    case 2: return launch_stream<T, KIND, 32, 8, 2, 2>(a, st, num_sms);
    case 3: return launch_stream<T, KIND, 32, 4, 4, 2>(a, st, num_sms);
    case 4: return launch_stream<T, KIND, 64, 4, 2, 2>(a, st, num_sms);
    case 6: return launch_stream<T, KIND, 64, 4, 4, 2>(a, st, num_sms);
    case 7: return launch_stream<T, KIND, 128, 2, 4, 2>(a, st, num_sms);
    case 8: return launch_stream<T, KIND, 32, 8, 1, 3, true>(a, st, num_sms);
    case 9:  // falls back to 8 where its staged tiles exceed shared memory
        if constexpr (stream_smem<T, KIND, 32, 8, 2, 2, true>() <= 227 * 1024)
            return launch_stream<T, KIND, 32, 8, 2, 2, true>(a, st, num_sms);
        else
            return launch_stream<T, KIND, 32, 8, 1, 3, true>(a, st, num_sms);
    case 5:
        if constexpr (sizeof(T) == 4) {
            if constexpr (R == 1) return launch_cfg<T, KIND, false, 64, 4, 8, 2>(a, st, num_sms);
            else return launch_cfg<T, KIND, false, 32, 8, 4, 2>(a, st, num_sms);
        } else {
            if constexpr (R == 1) return launch_cfg<T, KIND, false, 32, 8, 4, 2>(a, st, num_sms);
            else return launch_cfg<T, KIND, false, 32, 8, 2, 2>(a, st, num_sms);
        }
    default: return cudaErrorInvalidValue;
    }
}

// Adjoint sweep of the variable-coefficient kinds: the streaming kernel with
// the transposed operator (source-point coefficients prefetched in
// registers).  Variant 5 selects the register-staged plain kernel instead.
template <typename T, int KIND>
static cudaError_t launch_adjoint_var(const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    constexpr int R = KindTraits<KIND>::R;
    if (a.variant == 5) {
        if constexpr (sizeof(T) == 4) {
            if constexpr (R == 1) return launch_cfg<T, KIND, true, 64, 4, 8, 2>(a, st, num_sms);
            else return launch_cfg<T, KIND, true, 32, 8, 4, 2>(a, st, num_sms);
        } else {
            if constexpr (R == 1) return launch_cfg<T, KIND, true, 32, 8, 4, 2>(a, st, num_sms);
            else return launch_cfg<T, KIND, true, 32, 8, 2, 2>(a, st, num_sms);
        }
    }
    if constexpr (R == 1) return launch_stream<T, KIND, 32, 8, 2, 2, false, true>(a, st, num_sms);
    else return launch_stream<T, KIND, 32, 8, 1, 2, false, true>(a, st, num_sms);
}

template <typename T>
cudaError_t launch_plain(int kind, bool adjoint, const SweepArgs<T> &a, cudaStream_t st, int num_sms) {
    const int v = a.variant;
    switch (kind) {
    // the constant kinds are symmetric: their adjoint is the forward sweep
    case J7_CONST: return launch_forward<T, J7_CONST>(a, st, num_sms, v);
    case W25_CONST: return launch_forward<T, W25_CONST>(a, st, num_sms, v);
    case J7_VAR: return adjoint ? launch_adjoint_var<T, J7_VAR>(a, st, num_sms) : launch_forward<T, J7_VAR>(a, st, num_sms, v);
    case W25_VAR: return adjoint ? launch_adjoint_var<T, W25_VAR>(a, st, num_sms) : launch_forward<T, W25_VAR>(a, st, num_sms, v);
    case J25_VAR: return adjoint ? launch_adjoint_var<T, J25_VAR>(a, st, num_sms) : launch_forward<T, J25_VAR>(a, st, num_sms, v);
    case W25_ALPHA: return adjoint ? launch_adjoint_var<T, W25_ALPHA>(a, st, num_sms) : launch_forward<T, W25_ALPHA>(a, st, num_sms, v);
    default: return cudaErrorInvalidValue;
    }
}

template cudaError_t launch_plain<double>(int, bool, const SweepArgs<double> &, cudaStream_t, int);

}  // namespace stc
