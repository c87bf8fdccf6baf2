// wavefront_f32.cu -- FP32 instances of the register wavefront passes.
#include "wavefront_impl.cuh"

namespace stc {

bool wavefront_supported(int kind, int dtype, int levels, const Geom &g) {
    if (kind != J7_CONST && kind != J7_VAR) return false;
    const int maxb = dtype == 1 ? 4 : 2;
    if (levels < 1 || levels > maxb) return false;
    const int V = kVec(dtype == 1 ? 4 : 8);
    return g.px % V == 0 && (int64_t)g.px * g.py < (int64_t)1 << 30;
}

template <typename T>
cudaError_t launch_wavefront(int kind, const BlockedArgs<T> &a, int tile, cudaStream_t st, int num_sms) {
    return launch_wavefront_impl<T>(kind, a, tile, st, num_sms);
}

template cudaError_t launch_wavefront<float>(int, const BlockedArgs<float> &, int, cudaStream_t, int);

bool wavefront_info_f32(int kind, int levels, int tile, int64_t *info) {
    return wavefront_info_impl<float>(kind, levels, tile, info);
}

}  // namespace stc
