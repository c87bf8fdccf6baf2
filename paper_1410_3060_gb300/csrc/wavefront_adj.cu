// wavefront_adj.cu -- FP32 and FP64 instances of the depth-2 adjoint passes of
// the register wavefront (a translation unit of their own, compiled in
// parallel with the forward instances).
#include "wavefront_impl.cuh"

namespace stc {

template <typename T>
cudaError_t launch_wavefront_adj(int kind, const BlockedArgs<T> &a, int tile, cudaStream_t st, int num_sms) {
    return launch_wavefront_adj_impl<T>(kind, a, tile, st, num_sms);
}

template cudaError_t launch_wavefront_adj<float>(int, const BlockedArgs<float> &, int, cudaStream_t, int);
template cudaError_t launch_wavefront_adj<double>(int, const BlockedArgs<double> &, int, cudaStream_t, int);

}  // namespace stc
