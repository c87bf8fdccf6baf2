// plainv_f32.cu -- FP32 instances of the vectorised plain sweep of the 25-point kinds.
#include "plainv_impl.cuh"
#include "blk25_impl.cuh"

namespace stc {

bool plainv_supported_f32(int kind, const Geom &g) { return plainv_supported<float>(kind, g); }
unsigned int plainv_timeouts_f32() { return plainv_read_timeouts(); }
bool plainv_info_f32(int kind, int variant, int64_t *info) { return plainv_info<float>(kind, variant, info); }

template cudaError_t launch_plainv_kind<float>(int, bool, const SweepArgs<float> &, int, cudaStream_t, int);

bool blk25_supported_f32(int kind, int levels, const Geom &g) { return blk25_supported(kind, levels, g); }
bool blk25_info_f32(int kind, int64_t *info) { return blk25_info(kind, info); }
cudaError_t launch_blk25_f32(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms) {
    return launch_blk25(kind, a, st, num_sms);
}
cudaError_t launch_blk25_adj_f32(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms) {
    return launch_blk25(kind, a, st, num_sms, true);
}

}  // namespace stc
