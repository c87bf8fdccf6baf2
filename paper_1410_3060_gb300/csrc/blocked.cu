// blocked.cu -- temporally blocked passes (placeholder: none yet).
#include "blocked.cuh"

namespace stc {

bool blocked_supported(int, int, int) { return false; }
int blocked_default_levels(int, int) { return 1; }
template <typename T>
cudaError_t launch_blocked(int, const BlockedArgs<T> &, cudaStream_t, int, int) { return cudaErrorNotSupported; }
template cudaError_t launch_blocked<float>(int, const BlockedArgs<float> &, cudaStream_t, int, int);
template cudaError_t launch_blocked<double>(int, const BlockedArgs<double> &, cudaStream_t, int, int);

}  // namespace stc
