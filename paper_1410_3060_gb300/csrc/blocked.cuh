// blocked.cuh -- temporally blocked passes (several time levels per sweep).
#pragma once
#include "common.cuh"

namespace stc {

template <typename T>
struct BlockedArgs {
    const T *u_prev;     // level t-1 (second-order kinds)
    const T *u;          // level t
    T *out_prev;         // receives level t+levels-1, or nullptr
    T *out;              // receives level t+levels
    const T *W;          // coefficient stack
    T *trace;            // trace rows of levels t+1..t+levels ([levels][ny][nx]) or nullptr
    Scalars s;
    Geom g;
    T *bands[8];         // diamond edge bands of levels 1..levels-1 (padded fields)
    int rcv_z;
    int levels;
    int zchunk;
    int wA;              // phase-A tile height (diamond scheme)
    unsigned long long *dbg;   // debug builds: first bad store index + 1 (nullptr otherwise)
    int wait_limit;      // polls of a bounded mbarrier wait (TMA-staged passes)
    // adjoint passes: residual plane [ny][nx] added to level 1 on plane
    // rcv_z (nullptr: none); level k's plane is inject + (k-1) * inject_step
    const T *inject;
    int64_t inject_step;
};

bool blocked_supported(int kind, int dtype, int levels);
int blocked_default_levels(int kind, int dtype);
// padded fields of band scratch a pass of `levels` levels needs
int blocked_scratch_levels(int levels);
template <typename T>
cudaError_t launch_blocked(int kind, const BlockedArgs<T> &a, cudaStream_t st, int num_sms, int scheme);

}  // namespace stc
