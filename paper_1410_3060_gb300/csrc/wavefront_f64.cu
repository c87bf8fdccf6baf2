// wavefront_f64.cu -- FP64 instances of the register wavefront passes.
#include "wavefront_impl.cuh"

namespace stc {

template <typename T>
cudaError_t launch_wavefront(int kind, const BlockedArgs<T> &a, int tile, cudaStream_t st, int num_sms) {
    return launch_wavefront_impl<T>(kind, a, tile, st, num_sms);
}

template cudaError_t launch_wavefront<double>(int, const BlockedArgs<double> &, int, cudaStream_t, int);

bool wavefront_info_f64(int kind, int levels, int tile, int64_t *info) {
    return wavefront_info_impl<double>(kind, levels, tile, info);
}

}  // namespace stc
