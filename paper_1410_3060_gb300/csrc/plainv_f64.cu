// plainv_f64.cu -- FP64 instances of the vectorised plain sweep of the 25-point kinds.
#include "plainv_impl.cuh"

namespace stc {

bool plainv_supported_f64(int kind, const Geom &g) { return plainv_supported<double>(kind, g); }
unsigned int plainv_timeouts_f64() { return plainv_read_timeouts(); }
bool plainv_info_f64(int kind, int variant, int64_t *info) { return plainv_info<double>(kind, variant, info); }

template cudaError_t launch_plainv_kind<double>(int, bool, const SweepArgs<double> &, int, cudaStream_t, int);

}  // namespace stc
