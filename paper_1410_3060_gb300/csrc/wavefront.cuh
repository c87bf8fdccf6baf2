// wavefront.cuh -- register wavefront passes (B time levels per sweep, B >= 1)
// with warp-shuffle x neighbours and overlapped tiles.
#pragma once
#include "blocked.cuh"

namespace stc {

// Whether the register wavefront serves this kind / dtype / depth and the
// plan's geometry (vector width: the padded row length must be a multiple of
// the elements per thread).
bool wavefront_supported(int kind, int dtype, int levels, const Geom &g);
// Tile variant of the register wavefront (0 = default of the kind / dtype).
template <typename T>
cudaError_t launch_wavefront(int kind, const BlockedArgs<T> &a, int tile, cudaStream_t st, int num_sms);
// Adjoint pass of depth 2 (a.levels == 2) of the 7-point kinds: lam^{t+1}
// in a.u, level 1 (lam^t) into a.out_prev, level 2 (lam^{t-1}) into a.out,
// residual planes a.inject / a.inject + a.inject_step on plane a.rcv_z;
// tiles 0-3 (wavefront_adj.cu).
template <typename T>
cudaError_t launch_wavefront_adj(int kind, const BlockedArgs<T> &a, int tile, cudaStream_t st, int num_sms);
// Resources of a pass configuration (info[0..5]: dynamic shared memory bytes,
// threads, computed x / y extent, owned x / y extent); false if not served.
bool wavefront_info_f32(int kind, int levels, int tile, int64_t *info);
bool wavefront_info_f64(int kind, int levels, int tile, int64_t *info);

// Two-level TMA-staged pass of the 13-array 25-point kinds, FP32 (scheme 4;
// blk25_impl.cuh).
bool blk25_supported_f32(int kind, int levels, const Geom &g);
cudaError_t launch_blk25_f32(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms);
// Its adjoint (W25_VAR, J25_VAR): lam^{t+1} in a.u, lam^{t+2} in a.u_prev
// (wave kind), level 1 into a.out_prev, level 2 into a.out, residual planes
// a.inject / a.inject + a.inject_step on plane a.rcv_z.
cudaError_t launch_blk25_adj_f32(int kind, const BlockedArgs<float> &a, cudaStream_t st, int num_sms);
bool blk25_info_f32(int kind, int64_t *info);

}  // namespace stc
