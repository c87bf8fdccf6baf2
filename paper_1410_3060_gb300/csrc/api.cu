// api.cu -- the C ABI of libstencil.so (include/stencil.h): plans, argument
// validation, the time-loop program (which passes run on which buffers) and
// the forward / adjoint drivers.
//
// Time loop (paper Sect. 3.1: T sweeps over two time copies; Sect. 4: a
// temporally blocked pass applies several time levels per sweep).  The
// driver splits T into passes and assigns buffers so that on return the
// caller's (u_prev, u) hold (u^{T-1}, u^T) without extra copies in the
// common case:
//  * second-order kinds: a plain pass updates in place (u^{t+1} overwrites
//    u^{t-1}, the paper's two-copy scheme) and swaps the roles of the two
//    buffers; a blocked pass reads the pair and writes the new pair into the
//    other buffer set (caller's pair <-> plan scratch pair), choosing the
//    order so that the last one lands as (u_prev, u);
//  * first-order kinds: every pass reads the current buffer and writes the
//    other caller buffer; the last pass is a plain step so that the buffer
//    it reads holds u^{T-1}; an odd pass count starts with one copy.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/stencil.h"
#include "plain.cuh"
#include "blocked.cuh"
#include "wavefront.cuh"

using namespace stc;

namespace stc {
// Default forward tile variant per kind and dtype (0 = FP64, 1 = FP32): the
// variant measured fastest on GB300 at 512^3 (see the tile sweep in the
// design notes).
int default_variant(int kind, int dtype) {
    if (dtype == 1) {  // FP32 (sweep at 512^3, T = 8)
        switch (kind) {
        case J7_CONST: return 7;               // 128 x 8 tiles
        case J7_VAR: return 3;                 // 32 x 16, 4 rows per thread
        case W25_CONST: case W25_ALPHA: return 9;  // 32 x 16, staged u^{t-1}
        default: return 4;                     // W25_VAR, J25_VAR: 64 x 8
        }
    }
    switch (kind) {    // FP64 (bound by the FP64 pipe)
    case J7_CONST: return 3;
    case J7_VAR: case W25_CONST: case W25_ALPHA: return 8;  // staged per-point inputs
    default: return 1;                         // 32 x 8, one row per thread
    }
}
}  // namespace stc

namespace {

thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return STENCIL_ECUDA;
}

struct Op {
    int op, levels, in_p, in_c, out_p, out_c;
};

enum { BUF_A = 0, BUF_B = 1, BUF_S1 = 2, BUF_S2 = 3 };

// The pass program of T steps with block depth b (see the file comment).
// Split n levels into passes of at most b levels each, using only depths the
// blocked kernels provide (ok(L)); anything left becomes plain 1-level passes.
template <typename OK>
void split_levels(std::vector<int> &L, int64_t n, int b, OK ok) {
    while (n > 0) {
        int take = (int)std::min<int64_t>(n, b);
        while (take > 1 && !ok(take)) --take;
        L.push_back(take);
        n -= take;
    }
}

template <typename OK>
std::vector<Op> build_program(int kind, int64_t T, int b, OK ok) {
    std::vector<Op> ops;
    if (T <= 0) return ops;
    if (b < 1) b = 1;
    std::vector<int> L;
    const bool wave = kind_wave(kind);
    if (wave) {
        if (T == 1) {
            ops.push_back({0, 1, BUF_A, BUF_B, BUF_S1, BUF_S2});
            ops.push_back({1, 0, -1, BUF_S1, -1, BUF_A});
            ops.push_back({1, 0, -1, BUF_S2, -1, BUF_B});
            return ops;
        }
        split_levels(L, T, b, ok);
        // a pass of >= 2 levels moves the pair to the other buffer set; a
        // 1-level pass may be an in-place update (stays) or a move
        std::vector<bool> move(L.size());
        auto count = [&]() { int c = 0; for (bool m : move) c += m; return c; };
        auto last_single = [&](bool as_move) {
            for (int i = (int)L.size() - 1; i >= 0; --i)
                if (L[i] == 1 && move[i] == as_move) return i;
            return -1;
        };
        for (size_t i = 0; i < L.size(); ++i) move[i] = L[i] >= 2;
        if (count() % 2 == 1) {
            if (last_single(false) < 0) {
                // no 1-level pass: peel one level off the last pass
                const int v = L.back();
                L.pop_back();
                move.pop_back();
                std::vector<int> head;
                split_levels(head, v - 1, v - 1, ok);
                for (int h : head) { L.push_back(h); move.push_back(h >= 2); }
                L.push_back(1);
                move.push_back(false);
            }
            if (count() % 2 == 1) move[last_single(false)] = true;
        }
        if (count() == 0 && T % 2 == 1) {
            // all in place with an odd count would leave the pair swapped:
            // route two single steps through the scratch pair
            move[last_single(false)] = true;
            move[last_single(false)] = true;
        }
        int P = BUF_A, C = BUF_B;
        bool in_user = true;
        for (size_t i = 0; i < L.size(); ++i) {
            if (!move[i]) {
                ops.push_back({0, L[i], P, C, -1, P});
                std::swap(P, C);
            } else {
                int op_, oc;
                if (in_user) {
                    op_ = BUF_S1; oc = BUF_S2;
                } else {
                    int f = 0;
                    for (size_t k = i + 1; k < L.size(); ++k) f += !move[k];
                    if (f % 2 == 0) { op_ = BUF_A; oc = BUF_B; } else { op_ = BUF_B; oc = BUF_A; }
                }
                ops.push_back({0, L[i], P, C, op_, oc});
                P = op_; C = oc;
                in_user = !in_user;
            }
        }
    } else {
        if (b == 1) {
            L.assign((size_t)T, 1);
        } else {
            split_levels(L, T - 1, b, ok);
            L.push_back(1);
        }
        int C = BUF_B;
        if (L.size() % 2 == 1) {
            ops.push_back({1, 0, -1, BUF_B, -1, BUF_A});
            C = BUF_A;
        }
        for (size_t i = 0; i < L.size(); ++i) {
            const int out = (C == BUF_A) ? BUF_B : BUF_A;
            ops.push_back({0, L[i], C == BUF_A ? BUF_B : BUF_A, C, -1, out});
            C = out;
        }
    }
    return ops;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

}  // namespace

struct stencil_plan_s {
    int kind, dtype, R;
    Geom g;
    int device, num_sms;
    int time_block;   // 0 = default
    int scheme;       // 0 = default
    size_t elem, field_bytes;
    void *scratch[2];
    void *bands[8];   // diamond edge bands of the blocked passes
    int nbands;
    int variant;      // forward sweep tile variant (0 = default)
    int grad_batch;   // adjoint steps per FP64 gradient update
    void *gring[2 * GRAD_MAX_STEPS + 2];  // adjoint levels of two gradient batches
    cudaStream_t grad_stream;         // gradient batches run here, overlapping the next batch's sweeps
    cudaEvent_t ev_sweeps, ev_grad[2];
    int ngring;
    double *partials;
    int npartials;
    int wait_limit;        // polls of a bounded mbarrier wait (0 = default)
    int skip_plane;        // test hook of the bounded waits (SKIP_NONE = off)
    int adj_tb;            // levels per adjoint pass (0 = default)
    uint64_t timeouts_seen;   // device timeout counters at the last stencil_check
    unsigned long long *dbg;  // debug builds: first out-of-interior store index + 1 of the plan's sweeps
    // CUDA graph of the forward pass program (STENCIL_OPT_GRAPH)
    int graph;
    cudaStream_t cap_stream;
    cudaGraphExec_t gexec;
    bool gvalid;
    struct GraphKey {
        void *up, *u, *trace;
        const void *arrays;
        double w[8];
        int nw;
        int64_t T, rcv_z;
        int tb, scheme, variant;
        bool operator==(const GraphKey &o) const {
            if (up != o.up || u != o.u || trace != o.trace || arrays != o.arrays || nw != o.nw || T != o.T ||
                rcv_z != o.rcv_z || tb != o.tb || scheme != o.scheme || variant != o.variant)
                return false;
            for (int i = 0; i < nw; ++i)
                if (w[i] != o.w[i]) return false;
            return true;
        }
    } gkey;
};

namespace {

// FP32 7-point plans whose geometry the register wavefront serves default
// to it (measured fastest on GB300 at 512^3, T = 64: depth 3 with 64x64
// tiles for the constant kind, 898 GLUP/s; depth 2 with 64x32 tiles of 2
// rows per thread and the shared coefficient ring for the variable kind,
// 265); all other plans to the shared-memory kernels.
bool wavefront_default(const stencil_plan_s *p) {
    return p->dtype == 1 && (p->kind == J7_CONST || p->kind == J7_VAR) &&
           wavefront_supported(p->kind, p->dtype, 1, p->g);
}

// Register wavefront tile of a tile variant: 10-12 -> tiles 1-3 (64-column
// tiles), 17 -> tile 4 (FP32, 128-column tile of 4 points per thread row);
// 0 if the variant names no wavefront tile.
int wf_tile(int variant) {
    if (variant >= 10 && variant <= 12) return variant - 9;
    if (variant == 17) return 4;
    return 0;
}

int plan_scheme(const stencil_plan_s *p) {
    if (p->scheme) return p->scheme;
    return wavefront_default(p) ? 3 : 2;
}

// Default tile variant: the register wavefront tiles for FP32 7-point plans,
// the TMA-staged vectorised 25-point sweep where the geometry allows it
// (measured at 512^3: FP32 W25_CONST 448 vs 274 GLUP/s for the best
// streaming tile, W25_VAR 105 vs 76; FP64 W25_VAR 20.6 vs 18.6; FP64
// W25_CONST is FP64-bound either way and keeps the streaming kernel), else
// the streaming-kernel default.
int plan_variant(const stencil_plan_s *p) {
    if (p->variant) return p->variant;
    if (wavefront_default(p)) return p->kind == J7_CONST ? 12 : 11;
    const bool vec = p->dtype == 1 ? plainv_supported_f32(p->kind, p->g) : plainv_supported_f64(p->kind, p->g);
    if (vec) {
        const bool arrays13 = p->kind == W25_VAR || p->kind == J25_VAR;
        if (arrays13) return 16;
        // FP32 at 512^3: constant wave 449 (15) vs 414 (16) GLUP/s; alpha-array
        // wave 332 (16) vs 292 (15)
        if (p->dtype == 1) return p->kind == W25_ALPHA ? 16 : 15;
    }
    return default_variant(p->kind, p->dtype);
}

int default_time_block(const stencil_plan_s *p) {
    if (plan_scheme(p) == 3 && wavefront_default(p)) return p->kind == J7_CONST ? 3 : 2;
    return blocked_default_levels(p->kind, p->dtype);
}

// The register wavefront serves a blocked pass of scheme 3 (and a plain
// pass of tile variant 10-12) when it supports the kind, dtype, depth and
// geometry; the shared-memory blocked kernels serve schemes 1 and 2.
bool pass_supported(const stencil_plan_s *p, int levels) {
    if (plan_scheme(p) == 3) return wavefront_supported(p->kind, p->dtype, levels, p->g);
    if (plan_scheme(p) == 4) return p->dtype == 1 && blk25_supported_f32(p->kind, levels, p->g);
    return blocked_supported(p->kind, p->dtype, levels);
}

// Adjoint passes of depth 2 (both levels written): the register
// wavefront's adjoint for the 7-point kinds where the wavefront serves a
// forward pass of depth 2 on the plan's geometry; the two-level pass's
// adjoint for the 13-array kinds in FP32 where it serves the forward.
bool adj_pass_supported(const stencil_plan_s *p) {
    if (p->kind == J7_CONST || p->kind == J7_VAR) return wavefront_supported(p->kind, p->dtype, 2, p->g);
    return (p->kind == W25_VAR || p->kind == J25_VAR) && p->dtype == STENCIL_F32 &&
           blk25_supported_f32(p->kind, 2, p->g);
}

// Default adjoint depth: 2 for the FP32 7-point kinds (measured at 512^3,
// T = 64: J7_VAR 259 vs 129 GLUP/s, J7_CONST 789 vs 584), else 1 (FP64 is
// bound by the FP64 pipe: 54.0 vs 55.3 for J7_VAR; the 13-array kinds' pass
// gathers 29 coefficient vectors per point vector and is slower than their
// one-level adjoint).
int effective_adj_block(const stencil_plan_s *p) {
    const bool r1 = p->kind == J7_CONST || p->kind == J7_VAR;
    const int b = p->adj_tb > 0 ? p->adj_tb : (p->dtype == STENCIL_F32 && r1 ? 2 : 1);
    return (b == 2 && adj_pass_supported(p)) ? 2 : 1;
}

// Tile of the adjoint passes: the plan's register wavefront tile variant
// 10-12 when one is set, else the measured best at 512^3 FP32: J7_VAR the
// 64 x 32 tile of 2 rows per thread (259 GLUP/s, its gathered coefficients
// reused through a shared slot; 197 with 4 rows per thread, 140 for
// 64 x 64), J7_CONST 64 x 64 (789 vs 697 and 786).
int adj_tile(const stencil_plan_s *p) {
    const int t = wf_tile(p->variant);
    if (t >= 1 && t <= 3) return t;
    return p->kind == J7_VAR ? 2 : 3;
}

int effective_time_block(const stencil_plan_s *p) {
    int b = p->time_block > 0 ? p->time_block : default_time_block(p);
    if (b > 1 && !pass_supported(p, b)) b = 1;
    return b;
}

int check_coeffs(const stencil_plan_s *p, const stencil_coeffs_t *c) {
    const int nw = kind_weights(p->kind), na = kind_arrays(p->kind);
    if (nw > 0 && (!c || !c->w || c->nw != nw)) return STENCIL_EINVAL;
    if (na > 0 && (!c || !c->arrays || !aligned16(c->arrays))) return STENCIL_EINVAL;
    return STENCIL_OK;
}

Scalars fold_scalars(int kind, const stencil_coeffs_t *c) {
    Scalars s;
    memset(&s, 0, sizeof(s));
    if (kind == J7_CONST) {
        s.c[0] = c->w[0];
        s.c[1] = c->w[1];
    } else if (kind == W25_CONST) {
        const double al = c->w[0];
        s.c[0] = 2.0 + al * c->w[1];
        for (int r = 1; r <= 4; ++r) s.c[r] = al * c->w[1 + r];
    } else if (kind == W25_ALPHA) {
        for (int r = 0; r <= 4; ++r) s.c[r] = c->w[r];
    }
    return s;
}

bool overlap(const void *a, const void *b, size_t n) {
    const uintptr_t x = (uintptr_t)a, y = (uintptr_t)b;
    return x < y + n && y < x + n;
}

// One plain (one-level) sweep: the register wavefront at depth 1 for tile
// variants >= 10 where it serves the kind and geometry (forward only), else
// the plain kernels.
template <typename T>
cudaError_t plain_step(stencil_plan_s *p, bool adjoint, const Scalars &s, const stencil_coeffs_t *coeffs,
                       const void *in_p, const void *in_c, void *out, T *trace, const T *inject, int64_t rcv_z,
                       cudaStream_t st) {
    int variant = plan_variant(p);
    // a one-level pass of a default FP32 7-point constant plan runs the
    // 64 x 32 tile of 2 rows per thread (measured at 512^3: 599 vs 557 GLUP/s
    // for the 64 x 64 tile its blocked passes use)
    if (!p->variant && variant == 12 && p->kind == J7_CONST && p->dtype == 1) variant = 11;
    if (!adjoint && wf_tile(variant) && wavefront_supported(p->kind, p->dtype, 1, p->g)) {
        BlockedArgs<T> w;
        memset(&w, 0, sizeof(w));
        w.u = (const T *)in_c;
        w.out = (T *)out;
        w.W = coeffs ? (const T *)coeffs->arrays : nullptr;
        w.s = s;
        w.g = p->g;
        w.rcv_z = (int)rcv_z;
        w.trace = trace;
        w.levels = 1;
        w.dbg = p->dbg;
        return launch_wavefront<T>(p->kind, w, wf_tile(variant), st, p->num_sms);
    }
    SweepArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.u_prev = (const T *)in_p;
    a.u = (const T *)in_c;
    a.out = (T *)out;
    a.W = coeffs ? (const T *)coeffs->arrays : nullptr;
    a.s = s;
    a.g = p->g;
    a.rcv_z = (int)rcv_z;
    a.trace = trace;
    a.inject = inject;
    a.wait_limit = p->wait_limit;
    a.skip_plane = p->skip_plane;
    a.dbg = p->dbg;
    // the vectorised 25-point sweep (forward and adjoint)
    if (variant >= 13 && variant <= 16 && (!adjoint || kind_radius(p->kind) == 4) &&
        (p->dtype == 1 ? plainv_supported_f32(p->kind, p->g) : plainv_supported_f64(p->kind, p->g)))
        return launch_plainv_kind<T>(p->kind, adjoint, a, variant, st, p->num_sms);
    a.variant = variant < 10 ? variant : 0;  // 10+: register wavefront / vectorised tiles
    return launch_plain<T>(p->kind, adjoint, a, st, p->num_sms);
}

// One depth-2 adjoint pass: lam^{t+1} (in, with lam^{t+2} in in_p for the
// second-order kinds) gives lam^t (into out1, if not null) and lam^{t-1}
// (into out2); inj1 is the residual plane of the first level (the second
// level's is the plane before it in the residual stack), added on plane
// rcv_z.
template <typename T>
cudaError_t adjoint_pair(stencil_plan_s *p, const Scalars &s, const stencil_coeffs_t *coeffs, const void *in_p,
                         const void *in, void *out1, void *out2, const T *inj1, int64_t rcv_z, cudaStream_t st) {
    BlockedArgs<T> a;
    memset(&a, 0, sizeof(a));
    a.u_prev = (const T *)in_p;   // lam^{t+2} (second-order kinds)
    a.u = (const T *)in;
    a.out_prev = (T *)out1;
    a.out = (T *)out2;
    a.W = coeffs ? (const T *)coeffs->arrays : nullptr;
    a.s = s;
    a.g = p->g;
    a.rcv_z = (int)rcv_z;
    a.levels = 2;
    a.dbg = p->dbg;
    a.wait_limit = p->wait_limit;
    a.inject = inj1;
    a.inject_step = -(int64_t)p->g.nx * p->g.ny;
    if (p->kind == J7_CONST || p->kind == J7_VAR) return launch_wavefront_adj<T>(p->kind, a, adj_tile(p), st, p->num_sms);
    if constexpr (sizeof(T) == 4) return launch_blk25_adj_f32(p->kind, a, st, p->num_sms);
    return cudaErrorNotSupported;
}

template <typename T>
int run_program(stencil_plan_s *p, void *pair_p, void *pair_c, const stencil_coeffs_t *coeffs, int64_t nsteps,
                 cudaStream_t st, bool adjoint, void *trace, const void *inject, int64_t rcv_z,
                 const void *const *fwd_states, double *grad) {
    // adjoint: the caller sets time_block to the adjoint depth (1 or 2)
    const int b = adjoint ? p->time_block : effective_time_block(p);
    const std::vector<Op> ops = build_program(p->kind, nsteps, b, [&](int L) {
        return adjoint ? (L == 2 && adj_pass_supported(p)) : pass_supported(p, L);
    });
    void *buf[4] = {pair_p, pair_c, p->scratch[0], p->scratch[1]};
    const Scalars s = fold_scalars(p->kind, coeffs);
    const int64_t plane = (int64_t)p->g.nx * p->g.ny;
    int64_t t = 0;  // steps done
    for (const Op &o : ops) {
        if (o.op == 1) {
            cudaError_t e = cudaMemcpyAsync(buf[o.out_c], buf[o.in_c], p->field_bytes, cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) return cuda_fail(e);
            continue;
        }
        if (o.levels == 1) {
            // step index of this level: forward writes trace[t]; the adjoint
            // step j = t + 1 produces lam^{m-j} and uses fwd_states[nsteps-j]
            // and residual[nsteps-j]
            const int64_t j = t + 1;
            if (adjoint && grad) {
                GradArgs<T> ga;
                memset(&ga, 0, sizeof(ga));
                ga.u[0] = (const T *)fwd_states[nsteps - j];
                ga.lam[0] = (const T *)buf[o.in_c];
                ga.grad = grad;
                ga.s = s;
                if (p->kind == W25_ALPHA)
                    for (int r = 0; r <= 4; ++r) ga.s.c[r] = coeffs->w[r];
                ga.g = p->g;
                ga.nsteps = 1;
                cudaError_t e = launch_grad<T>(p->kind, ga, st);
                if (e != cudaSuccess) return cuda_fail(e);
            }
            if (o.out_p >= 0) {
                cudaError_t e = cudaMemcpyAsync(buf[o.out_p], buf[o.in_c], p->field_bytes, cudaMemcpyDeviceToDevice, st);
                if (e != cudaSuccess) return cuda_fail(e);
            }
            cudaError_t e = plain_step<T>(p, adjoint, s, coeffs, buf[o.in_p], buf[o.in_c], buf[o.out_c],
                                          (!adjoint && trace) ? (T *)trace + t * plane : nullptr,
                                          (adjoint && inject) ? (const T *)inject + (nsteps - j) * plane : nullptr,
                                          rcv_z, st);
            if (e != cudaSuccess) return cuda_fail(e);
        } else if (adjoint) {
            // depth-2 adjoint pass: steps j = t+1 and t+2 (residual planes
            // nsteps-j and nsteps-j-1); level 1 is kept where the program
            // needs it (the second-order kinds)
            if (o.levels != 2 || !adj_pass_supported(p)) return STENCIL_EUNSUPPORTED;
            const int64_t j = t + 1;
            cudaError_t e = adjoint_pair<T>(p, s, coeffs, buf[o.in_p], buf[o.in_c], o.out_p >= 0 ? buf[o.out_p] : nullptr,
                                            buf[o.out_c], inject ? (const T *)inject + (nsteps - j) * plane : nullptr,
                                            rcv_z, st);
            if (e != cudaSuccess) return cuda_fail(e);
        } else {
            BlockedArgs<T> a;
            memset(&a, 0, sizeof(a));
            a.u_prev = (const T *)buf[o.in_p];
            a.u = (const T *)buf[o.in_c];
            a.out_prev = o.out_p >= 0 ? (T *)buf[o.out_p] : nullptr;
            a.out = (T *)buf[o.out_c];
            a.W = coeffs ? (const T *)coeffs->arrays : nullptr;
            a.s = s;
            a.g = p->g;
            a.rcv_z = (int)rcv_z;
            a.trace = trace ? (T *)trace + t * plane : nullptr;
            a.levels = o.levels;
            a.dbg = p->dbg;
            a.wait_limit = p->wait_limit;
            cudaError_t e;
            const int scheme = plan_scheme(p), variant = plan_variant(p);
            if (scheme == 3) {
                e = launch_wavefront<T>(p->kind, a, wf_tile(variant), st, p->num_sms);
            } else if (scheme == 4) {
                if constexpr (sizeof(T) == 4) e = launch_blk25_f32(p->kind, a, st, p->num_sms);
                else return STENCIL_EUNSUPPORTED;
            } else {
                if (blocked_scratch_levels(o.levels) > p->nbands) return STENCIL_EUNSUPPORTED;
                for (int k = 1; k < o.levels; ++k) a.bands[k] = (T *)p->bands[k - 1];
                e = launch_blocked<T>(p->kind, a, st, p->num_sms, scheme);
            }
            if (e != cudaSuccess) return cuda_fail(e);
        }
        t += o.levels;
    }
    return STENCIL_OK;
}


// Forward T plain steps storing every state: step t reads
// (u^{t-1}, u^t) and writes u^{t+1} into states[t].
template <typename T>
int run_forward_states(stencil_plan_s *p, const void *u_prev, const void *u, const stencil_coeffs_t *coeffs,
                       int64_t nsteps, void *const *states, cudaStream_t st, void *trace, int64_t rcv_z) {
    const Scalars s = fold_scalars(p->kind, coeffs);
    const int64_t plane = (int64_t)p->g.nx * p->g.ny;
    // 7-point kinds whose plan runs register wavefront passes of depth >= 2:
    // a depth-2 pass writes both of its levels (and the trace of each), so
    // one pass gives two consecutive states
    const bool pairs = plan_scheme(p) == 3 && effective_time_block(p) >= 2 && !kind_wave(p->kind) &&
                       wavefront_supported(p->kind, p->dtype, 2, p->g);
    for (int64_t t = 0; t < nsteps;) {
        const void *ip = t >= 2 ? states[t - 2] : (t == 1 ? u : u_prev);
        const void *ic = t >= 1 ? states[t - 1] : u;
        cudaError_t e;
        if (pairs && t + 1 < nsteps) {
            BlockedArgs<T> a;
            memset(&a, 0, sizeof(a));
            a.u_prev = (const T *)ip;
            a.u = (const T *)ic;
            a.out_prev = (T *)states[t];
            a.out = (T *)states[t + 1];
            a.W = coeffs ? (const T *)coeffs->arrays : nullptr;
            a.s = s;
            a.g = p->g;
            a.rcv_z = (int)rcv_z;
            a.trace = trace ? (T *)trace + t * plane : nullptr;
            a.levels = 2;
            a.dbg = p->dbg;
            a.wait_limit = p->wait_limit;
            e = launch_wavefront<T>(p->kind, a, wf_tile(plan_variant(p)), st, p->num_sms);
            t += 2;
        } else {
            e = plain_step<T>(p, false, s, coeffs, ip, ic, states[t], trace ? (T *)trace + t * plane : nullptr,
                              nullptr, rcv_z, st);
            t += 1;
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return STENCIL_OK;
}

// Adjoint with gradient batches: every adjoint level is written to a ring of
// 2G + 2 plan fields, and after every G steps one gradient launch sums the G
// terms lam^{n+1} * d(A u^n)/dA in FP64 registers and updates the gradient
// arrays once.  Step j (j = 1..T) produces lam^{m-j} into ring slot
// (j-1) mod (2G+2); its inputs lam^{m-j+1}, lam^{m-j+2} sit in the two
// previous slots (or the caller's pair).  2G + 2 slots are enough: batch b's
// gradient reads its G levels and the level before them while batch b+1's
// sweeps write the next G (G + 1 + G slots, plus one so that batch b+1's
// first sweep still sees both inputs), and the first sweep of batch b+2
// waits for batch b's gradient (ev_grad[b % 2]) before it overwrites them.
// The host program of the adjoint with gradient batches of G steps: ops in
// issue order,
//   {ADJ_WAIT, b, 0}  the caller's stream waits for gradient batch b - 2
//                     (event ev_grad[b % 2]) before batch b's first sweep;
//   {ADJ_SWEEP, j, n} the sweep of steps j .. j+n-1 (n = 1, or 2 when pairs
//                     are allowed and both steps fall into the batch),
//                     writing lam^{m-j} .. into ring slots (j-1) mod (2G+2);
//   {ADJ_GRAD, b, k}  gradient batch b over its k steps (ending at the
//                     last sweep), on the gradient stream.
// Host logic only (no CUDA call): stencil_adjoint_schedule exposes it.
enum { ADJ_WAIT = 0, ADJ_SWEEP = 1, ADJ_GRAD = 2 };
struct AdjOp {
    int op;
    int64_t a, b;
};
std::vector<AdjOp> adjoint_ring_program(int64_t nsteps, int G, bool pairs) {
    std::vector<AdjOp> ops;
    int64_t batch = 0, in_batch = 0;
    for (int64_t j = 1; j <= nsteps;) {
        // the first sweep of batch b >= 2 overwrites the levels batch b-2's gradient reads
        if (in_batch == 0 && batch >= 2) ops.push_back({ADJ_WAIT, batch, 0});
        const int n = (pairs && j + 1 <= nsteps && in_batch + 2 <= G) ? 2 : 1;
        ops.push_back({ADJ_SWEEP, j, n});
        in_batch += n;
        j += n;
        if (in_batch == G || j > nsteps) {
            ops.push_back({ADJ_GRAD, batch, in_batch});
            ++batch;
            in_batch = 0;
        }
    }
    return ops;
}

template <typename T>
int run_adjoint_ring(stencil_plan_s *p, void *lam_next, void *lam, const stencil_coeffs_t *coeffs, int64_t nsteps,
                     cudaStream_t st, const void *inject, int64_t rcv_z, const void *const *fwd_states,
                     double *grad) {
    // The adjoint levels live in a ring of 2G + 2 plan fields: the gradient
    // of batch b (levels bG .. bG+G-1) runs on the plan's gradient stream
    // while the sweeps of batch b+1 (which write levels up to (b+2)G) run on
    // the caller's stream; the sweeps of batch b+2 wait for it.  Gradient
    // batches stay in order on their stream (they update the same arrays).
    const int G = p->grad_batch, NSL = 2 * G + 2;
    const Scalars s = fold_scalars(p->kind, coeffs);
    const int64_t plane = (int64_t)p->g.nx * p->g.ny;
    auto level = [&](int64_t j) -> void * {  // buffer holding lam^{m-j}
        if (j == -1) return lam_next;
        if (j == 0) return lam;
        return p->gring[(j - 1) % NSL];
    };
    cudaError_t e = cudaSuccess;
    if (!p->grad_stream) {
        e = cudaStreamCreateWithFlags(&p->grad_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_sweeps, cudaEventDisableTiming);
        for (int i = 0; i < 2 && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&p->ev_grad[i], cudaEventDisableTiming);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    GradArgs<T> ga;
    memset(&ga, 0, sizeof(ga));
    ga.grad = grad;
    ga.s = s;
    if (p->kind == W25_ALPHA)
        for (int r = 0; r <= 4; ++r) ga.s.c[r] = coeffs->w[r];
    ga.g = p->g;
    int64_t batch = 0;   // batches launched
    for (const AdjOp &o : adjoint_ring_program(nsteps, G, effective_adj_block(p) == 2)) {
        if (o.op == ADJ_WAIT) {
            e = cudaStreamWaitEvent(st, p->ev_grad[o.a % 2], 0);
        } else if (o.op == ADJ_SWEEP) {
            const int64_t j = o.a;
            const T *inj = inject ? (const T *)inject + (nsteps - j) * plane : nullptr;
            // a depth-2 pass of steps j, j+1 writes lam^{m-j} and lam^{m-j-1}
            // into their ring slots
            if (o.b == 2)
                e = adjoint_pair<T>(p, s, coeffs, level(j - 2), level(j - 1), level(j), level(j + 1), inj, rcv_z, st);
            else
                e = plain_step<T>(p, true, s, coeffs, level(j - 2), level(j - 1), level(j), nullptr, inj, rcv_z, st);
            for (int64_t i = 0; i < o.b; ++i) {
                ga.u[ga.nsteps] = (const T *)fwd_states[nsteps - j - i];
                ga.lam[ga.nsteps] = (const T *)level(j - 1 + i);
                ++ga.nsteps;
            }
        } else {
            // the gradient stream starts this batch once its sweeps (and all
            // earlier work of the caller's stream) are done
            e = cudaEventRecord(p->ev_sweeps, st);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(p->grad_stream, p->ev_sweeps, 0);
            if (e == cudaSuccess) e = launch_grad<T>(p->kind, ga, p->grad_stream);
            if (e == cudaSuccess) e = cudaEventRecord(p->ev_grad[o.a % 2], p->grad_stream);
            batch = o.a + 1;
            ga.nsteps = 0;
        }
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // the caller's stream continues after every gradient batch
    if (batch > 0) {
        e = cudaStreamWaitEvent(st, p->ev_grad[(batch - 1) % 2], 0);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    // final pair (lam^{m-T+1}, lam^{m-T}) back into the caller's buffers
    if (level(nsteps - 1) != lam_next)
        e = cudaMemcpyAsync(lam_next, level(nsteps - 1), p->field_bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(lam, level(nsteps), p->field_bytes, cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

void free_bands(stencil_plan_s *p) {
    for (int i = 0; i < 8; ++i) {
        if (p->bands[i]) cudaFree(p->bands[i]);
        p->bands[i] = nullptr;
    }
    p->nbands = 0;
}

// Allocate the band buffers of the effective block depth (plan time only).
int ensure_bands(stencil_plan_s *p) {
    const int b = effective_time_block(p);
    const int need = (b > 1 && plan_scheme(p) != 3 && plan_scheme(p) != 4) ? blocked_scratch_levels(b) : 0;
    if (need <= p->nbands) return STENCIL_OK;
    free_bands(p);
    for (int i = 0; i < need; ++i) {
        cudaError_t e = cudaMalloc(&p->bands[i], p->field_bytes);
        if (e != cudaSuccess) {
            free_bands(p);
            g_last_cuda_error = (int)e;
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
    }
    p->nbands = need;
    return STENCIL_OK;
}

void free_gring(stencil_plan_s *p) {
    for (int i = 0; i < 2 * GRAD_MAX_STEPS + 2; ++i) {
        if (p->gring[i]) cudaFree(p->gring[i]);
        p->gring[i] = nullptr;
    }
    p->ngring = 0;
}

int ensure_gring(stencil_plan_s *p) {
    const int need = p->grad_batch > 1 ? 2 * p->grad_batch + 2 : 0;
    if (need <= p->ngring) return STENCIL_OK;
    free_gring(p);
    for (int i = 0; i < need; ++i) {
        cudaError_t e = cudaMalloc(&p->gring[i], p->field_bytes);
        if (e == cudaSuccess) e = cudaMemset(p->gring[i], 0, p->field_bytes);  // zero halo
        if (e != cudaSuccess) {
            free_gring(p);
            g_last_cuda_error = (int)e;
            cudaGetLastError();
            return STENCIL_ENOMEM;
        }
    }
    p->ngring = need;
    return STENCIL_OK;
}

void free_scratch(stencil_plan_s *p) {
    free_gring(p);
    free_bands(p);
    for (int i = 0; i < 2; ++i) {
        if (p->scratch[i]) cudaFree(p->scratch[i]);
        p->scratch[i] = nullptr;
    }
    if (p->partials) cudaFree(p->partials);
    p->partials = nullptr;
    if (p->dbg) cudaFree(p->dbg);
    p->dbg = nullptr;
}

}  // namespace

extern "C" {

static void drop_graph(stencil_plan_s *p) {
    if (p->gvalid) cudaGraphExecDestroy(p->gexec);
    p->gvalid = false;
}

int stencil_plan(stencil_plan_t *plan, int kind, int64_t nx, int64_t ny, int64_t nz, int radius, int dtype) {
    if (!plan) return STENCIL_EINVAL;
    *plan = nullptr;
    if (kind_radius(kind) < 0 || radius != kind_radius(kind)) return STENCIL_EINVAL;
    if (dtype != STENCIL_F64 && dtype != STENCIL_F32) return STENCIL_EINVAL;
    if (nx < 1 || ny < 1 || nz < 1) return STENCIL_EINVAL;
    const int64_t px = nx + 2 * radius, py = ny + 2 * radius, pz = nz + 2 * radius;
    if (px > (1 << 30) || py > (1 << 30) || pz > (1 << 30)) return STENCIL_EINVAL;
    if (px * py > ((int64_t)1 << 40) / pz) return STENCIL_EINVAL;
    stencil_plan_s *p = new stencil_plan_s;
    memset(p, 0, sizeof(*p));
    p->kind = kind;
    p->dtype = dtype;
    p->R = radius;
    p->g.nx = (int)nx; p->g.ny = (int)ny; p->g.nz = (int)nz;
    p->g.px = (int)px; p->g.py = (int)py; p->g.pz = (int)pz;
    p->g.sy = px;
    p->g.sz = px * py;
    p->g.nfield = px * py * pz;
    p->elem = dtype == STENCIL_F64 ? 8 : 4;
    p->grad_batch = 1;
    p->skip_plane = SKIP_NONE;
    p->timeouts_seen = (uint64_t)plainv_timeouts_f32() + plainv_timeouts_f64();
    p->field_bytes = (size_t)p->g.nfield * p->elem;
    cudaError_t e = cudaGetDevice(&p->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) { delete p; return cuda_fail(e); }
    // two scratch fields (second-order kinds move the state pair through
    // them) and the misfit partial sums
    const int nscratch = kind_wave(kind) ? 2 : 0;
    for (int i = 0; i < nscratch; ++i) {
        e = cudaMalloc(&p->scratch[i], p->field_bytes);
        if (e != cudaSuccess) { free_scratch(p); delete p; g_last_cuda_error = (int)e; cudaGetLastError(); return STENCIL_ENOMEM; }
        e = cudaMemset(p->scratch[i], 0, p->field_bytes);  // zero halo
        if (e != cudaSuccess) { free_scratch(p); delete p; return cuda_fail(e); }
    }
    p->npartials = 1024;
    e = cudaMalloc(&p->partials, p->npartials * sizeof(double));
    if (e != cudaSuccess) { free_scratch(p); delete p; g_last_cuda_error = (int)e; cudaGetLastError(); return STENCIL_ENOMEM; }
#ifdef STENCIL_DEBUG
    e = cudaMalloc(&p->dbg, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemset(p->dbg, 0, sizeof(unsigned long long));
    if (e != cudaSuccess) { free_scratch(p); delete p; g_last_cuda_error = (int)e; cudaGetLastError(); return STENCIL_ENOMEM; }
#endif
    const int st = ensure_bands(p);
    if (st != STENCIL_OK) { free_scratch(p); delete p; return st; }
    *plan = p;
    return STENCIL_OK;
}

int stencil_plan_set(stencil_plan_t p, int option, int64_t value) {
    if (!p) return STENCIL_EINVAL;
    drop_graph(p);   // any option may change the pass program or its scratch
    switch (option) {
    case STENCIL_OPT_TIME_BLOCK:
        if (value < 0 || value > 64) return STENCIL_EINVAL;
        if (value > 1 && !blocked_supported(p->kind, p->dtype, (int)value) &&
            !wavefront_supported(p->kind, p->dtype, (int)value, p->g) &&
            !(p->dtype == STENCIL_F32 && blk25_supported_f32(p->kind, (int)value, p->g)))
            return STENCIL_EUNSUPPORTED;
        p->time_block = (int)value;
        return ensure_bands(p);
    case STENCIL_OPT_SCHEME:
        if (value < 0 || value > 4) return STENCIL_EINVAL;
        p->scheme = (int)value;
        return ensure_bands(p);
    case STENCIL_OPT_VARIANT:
        if (value < 0 || value > 17) return STENCIL_EINVAL;
        if (value == 17 && p->dtype != STENCIL_F32) return STENCIL_EUNSUPPORTED;
        p->variant = (int)value;
        return STENCIL_OK;
    case STENCIL_OPT_GRAD_BATCH:
        if (value < 1 || value > GRAD_MAX_STEPS) return STENCIL_EINVAL;
        p->grad_batch = (int)value;
        return ensure_gring(p);
    case STENCIL_OPT_GRAPH:
        if (value < 0 || value > 1) return STENCIL_EINVAL;
        p->graph = (int)value;
        return STENCIL_OK;
    case STENCIL_OPT_WAIT_LIMIT:
        if (value < 0 || value > (1 << 30)) return STENCIL_EINVAL;
        p->wait_limit = (int)value;
        return STENCIL_OK;
    case STENCIL_OPT_ADJ_TIME_BLOCK:
        if (value < 0 || value > 2) return STENCIL_EINVAL;
        if (value == 2 && !adj_pass_supported(p)) return STENCIL_EUNSUPPORTED;
        p->adj_tb = (int)value;
        return STENCIL_OK;
    case STENCIL_OPT_TEST_SKIP_COPY:
        if (value < -1 || value >= p->g.nz) return STENCIL_EINVAL;
        p->skip_plane = value < 0 ? SKIP_NONE : (int)value;
        return STENCIL_OK;
    default:
        return STENCIL_EINVAL;
    }
}

int stencil_plan_get(stencil_plan_t p, int option, int64_t *value) {
    if (!p || !value) return STENCIL_EINVAL;
    switch (option) {
    case STENCIL_OPT_TIME_BLOCK: *value = effective_time_block(p); return STENCIL_OK;
    case STENCIL_OPT_SCHEME: *value = plan_scheme(p); return STENCIL_OK;
    case STENCIL_OPT_GRAD_BATCH: *value = p->grad_batch; return STENCIL_OK;
    case STENCIL_OPT_VARIANT:
        // the tile of the plan's passes (a default FP32 7-point constant plan
        // of one-level passes runs tile 11, see plain_step)
        *value = plan_variant(p);
        if (!p->variant && *value == 12 && p->kind == J7_CONST && p->dtype == 1 && effective_time_block(p) == 1)
            *value = 11;
        return STENCIL_OK;
    case STENCIL_OPT_GRAPH: *value = p->graph; return STENCIL_OK;
    case STENCIL_OPT_WAIT_LIMIT: *value = p->wait_limit > 0 ? p->wait_limit : WAIT_LIMIT_DEFAULT; return STENCIL_OK;
    case STENCIL_OPT_TEST_SKIP_COPY: *value = p->skip_plane == SKIP_NONE ? -1 : p->skip_plane; return STENCIL_OK;
    case STENCIL_OPT_ADJ_TIME_BLOCK: *value = effective_adj_block(p); return STENCIL_OK;
    case STENCIL_OPT_SCRATCH_BYTES:
        *value = (int64_t)((p->scratch[0] ? 2 * p->field_bytes : 0) + (p->nbands + p->ngring) * p->field_bytes +
                           p->npartials * sizeof(double));
        return STENCIL_OK;
    default: return STENCIL_EINVAL;
    }
}

void stencil_plan_destroy(stencil_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
    drop_graph(p);
    if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
    if (p->grad_stream) {
        cudaStreamDestroy(p->grad_stream);
        cudaEventDestroy(p->ev_sweeps);
        cudaEventDestroy(p->ev_grad[0]);
        cudaEventDestroy(p->ev_grad[1]);
    }
    free_scratch(p);
    delete p;
}

static int check_pair(stencil_plan_t p, void *a, void *b) {
    if (!a || !b || a == b) return STENCIL_EINVAL;
    if (!aligned16(a) || !aligned16(b)) return STENCIL_EINVAL;
    if (overlap(a, b, p->field_bytes)) return STENCIL_EINVAL;
    return STENCIL_OK;
}

int stencil_forward(stencil_plan_t p, void *u_prev, void *u, const stencil_coeffs_t *coeffs, int64_t T, void *stream,
                    void *trace, int64_t rcv_z) {
    if (!p || T < 0) return STENCIL_EINVAL;
    int st = check_pair(p, u_prev, u);
    if (st) return st;
    if ((st = check_coeffs(p, coeffs))) return st;
    if (trace && (rcv_z < 0 || rcv_z >= p->g.nz)) return STENCIL_EINVAL;
    if (T == 0) return STENCIL_OK;
    auto run = [&](cudaStream_t s) {
        if (p->dtype == STENCIL_F64)
            return run_program<double>(p, u_prev, u, coeffs, T, s, false, trace, nullptr, trace ? rcv_z : -1,
                                       nullptr, nullptr);
        return run_program<float>(p, u_prev, u, coeffs, T, s, false, trace, nullptr, trace ? rcv_z : -1, nullptr,
                                  nullptr);
    };
    if (!p->graph) return run((cudaStream_t)stream);
    // graph mode: the pass program of these arguments is captured once (on a
    // plan-owned stream, so the caller's stream may be the legacy default
    // stream) and replayed on the caller's stream
    stencil_plan_s::GraphKey key;
    memset(&key, 0, sizeof(key));
    key.up = u_prev;
    key.u = u;
    key.trace = trace;
    key.arrays = coeffs ? coeffs->arrays : nullptr;
    key.nw = coeffs && coeffs->w ? std::min<int>(coeffs->nw, 8) : 0;
    for (int i = 0; i < key.nw; ++i) key.w[i] = coeffs->w[i];
    key.T = T;
    key.rcv_z = trace ? rcv_z : -1;
    key.tb = effective_time_block(p);
    key.scheme = plan_scheme(p);
    key.variant = plan_variant(p);
    if (!p->gvalid || !(key == p->gkey)) {
        drop_graph(p);
        cudaError_t e = cudaSuccess;
        if (!p->cap_stream) e = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return cuda_fail(e);
        const int r = run(p->cap_stream);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(p->cap_stream, &graph);
        if (r != STENCIL_OK) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(e);
        e = cudaGraphInstantiate(&p->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) return cuda_fail(e);
        p->gvalid = true;
        p->gkey = key;
    }
    cudaError_t e = cudaGraphLaunch(p->gexec, (cudaStream_t)stream);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

int stencil_adjoint(stencil_plan_t p, void *lam_next, void *lam, const stencil_coeffs_t *coeffs, int64_t T,
                    void *stream, const void *const *fwd_states, const void *residual, int64_t rcv_z, double *grad) {
    if (!p || T < 0) return STENCIL_EINVAL;
    int st = check_pair(p, lam_next, lam);
    if (st) return st;
    if ((st = check_coeffs(p, coeffs))) return st;
    if (residual && (rcv_z < 0 || rcv_z >= p->g.nz)) return STENCIL_EINVAL;
    if (grad) {
        if (kind_arrays(p->kind) == 0) return STENCIL_EUNSUPPORTED;
        if (!aligned16(grad) || (T > 0 && !fwd_states)) return STENCIL_EINVAL;
        for (int64_t i = 0; i < T; ++i)
            if (!fwd_states[i]) return STENCIL_EINVAL;
    }
    if (T == 0) return STENCIL_OK;
    if (grad && p->grad_batch > 1) {
        if (p->dtype == STENCIL_F64)
            return run_adjoint_ring<double>(p, lam_next, lam, coeffs, T, (cudaStream_t)stream, residual,
                                            residual ? rcv_z : -1, fwd_states, grad);
        return run_adjoint_ring<float>(p, lam_next, lam, coeffs, T, (cudaStream_t)stream, residual,
                                       residual ? rcv_z : -1, fwd_states, grad);
    }
    // one-level passes, or depth-2 passes without a gradient (with a
    // gradient of batch 1 every level is summed before the next sweep)
    const int saved = p->time_block;
    p->time_block = grad ? 1 : effective_adj_block(p);
    int r;
    if (p->dtype == STENCIL_F64)
        r = run_program<double>(p, lam_next, lam, coeffs, T, (cudaStream_t)stream, true, nullptr, residual,
                                residual ? rcv_z : -1, fwd_states, grad);
    else
        r = run_program<float>(p, lam_next, lam, coeffs, T, (cudaStream_t)stream, true, nullptr, residual,
                               residual ? rcv_z : -1, fwd_states, grad);
    p->time_block = saved;
    return r;
}

int stencil_forward_states(stencil_plan_t p, const void *u_prev, const void *u, const stencil_coeffs_t *coeffs,
                           int64_t T, void *const *states, void *stream, void *trace, int64_t rcv_z) {
    if (!p || T < 0) return STENCIL_EINVAL;
    int st = check_pair(p, (void *)u_prev, (void *)u);
    if (st) return st;
    if ((st = check_coeffs(p, coeffs))) return st;
    if (trace && (rcv_z < 0 || rcv_z >= p->g.nz)) return STENCIL_EINVAL;
    if (T > 0 && !states) return STENCIL_EINVAL;
    for (int64_t t = 0; t < T; ++t) {
        if (!states[t] || !aligned16(states[t])) return STENCIL_EINVAL;
        if (overlap(states[t], u, p->field_bytes) || overlap(states[t], u_prev, p->field_bytes)) return STENCIL_EINVAL;
        if (t > 0 && overlap(states[t], states[t - 1], p->field_bytes)) return STENCIL_EINVAL;
        if (t > 1 && overlap(states[t], states[t - 2], p->field_bytes)) return STENCIL_EINVAL;
    }
    if (T == 0) return STENCIL_OK;
    if (p->dtype == STENCIL_F64)
        return run_forward_states<double>(p, u_prev, u, coeffs, T, states, (cudaStream_t)stream, trace,
                                          trace ? rcv_z : -1);
    return run_forward_states<float>(p, u_prev, u, coeffs, T, states, (cudaStream_t)stream, trace,
                                     trace ? rcv_z : -1);
}

int stencil_axpby(stencil_plan_t p, int64_t n, double alpha, const void *x, double beta, const void *y, void *out,
                  void *stream) {
    if (!p || !x || !y || !out || n < 0) return STENCIL_EINVAL;
    if (n == 0) return STENCIL_OK;
    cudaError_t e;
    if (p->dtype == STENCIL_F64)
        e = launch_axpby<double>(alpha, (const double *)x, beta, (const double *)y, (double *)out, n,
                                 p->num_sms, (cudaStream_t)stream);
    else
        e = launch_axpby<float>(alpha, (const float *)x, beta, (const float *)y, (float *)out, n,
                                p->num_sms, (cudaStream_t)stream);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

int stencil_fill_zero(void *ptr, int64_t bytes, void *stream) {
    if (!ptr || bytes < 0) return STENCIL_EINVAL;
    if (bytes == 0) return STENCIL_OK;
    cudaError_t e = cudaMemsetAsync(ptr, 0, (size_t)bytes, (cudaStream_t)stream);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

int stencil_misfit(stencil_plan_t p, const void *trace, const void *d, int64_t T, void *residual, double *loss,
                   void *stream) {
    if (!p || !trace || !d || !residual || !loss || T < 0) return STENCIL_EINVAL;
    const int64_t n = T * (int64_t)p->g.nx * p->g.ny;
    cudaError_t e;
    if (p->dtype == STENCIL_F64)
        e = launch_misfit<double>((const double *)trace, (const double *)d, (double *)residual, n, p->partials,
                                  p->npartials, loss, (cudaStream_t)stream);
    else
        e = launch_misfit<float>((const float *)trace, (const float *)d, (float *)residual, n, p->partials,
                                 p->npartials, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

int stencil_misfit_static(int dtype, const void *trace, const void *d, int64_t n, void *residual, double *loss,
                          void *stream) {
    if ((dtype != STENCIL_F64 && dtype != STENCIL_F32) || !trace || !d || !residual || !loss || n < 0)
        return STENCIL_EINVAL;
    if (n > STENCIL_MISFIT_STATIC_MAX_ELEMS) return STENCIL_EINVAL;  // needs more than the static partial sums
    static_assert(STENCIL_MISFIT_STATIC_MAX_ELEMS == MISFIT_STATIC_MAX_ELEMS, "header limit matches the array");
    cudaError_t e = misfit_static(dtype, trace, d, n, residual, loss, (cudaStream_t)stream);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

int stencil_schedule(int kind, int dtype, int64_t T, int b, int32_t *ops, int64_t max_ops, int64_t *n_ops) {
    if (kind_radius(kind) < 0 || (dtype != STENCIL_F64 && dtype != STENCIL_F32) || T < 0 || b < 1 || !n_ops ||
        (max_ops > 0 && !ops))
        return STENCIL_EINVAL;
    if (b > 1 && !blocked_supported(kind, dtype, b)) b = 1;
    const std::vector<Op> prog =
        build_program(kind, T, b, [&](int L) { return blocked_supported(kind, dtype, L); });
    *n_ops = (int64_t)prog.size();
    for (int64_t i = 0; i < (int64_t)prog.size() && i < max_ops; ++i) {
        const Op &o = prog[(size_t)i];
        const int32_t v[6] = {o.op, o.levels, o.in_p, o.in_c, o.out_p, o.out_c};
        memcpy(ops + 6 * i, v, sizeof(v));
    }
    return STENCIL_OK;
}

int stencil_adjoint_schedule(int64_t T, int grad_batch, int levels, int64_t *ops, int64_t max_ops,
                             int64_t *n_ops) {
    if (T < 0 || grad_batch < 1 || grad_batch > GRAD_MAX_STEPS || levels < 1 || levels > 2 || !n_ops ||
        (max_ops > 0 && !ops))
        return STENCIL_EINVAL;
    const std::vector<AdjOp> prog = adjoint_ring_program(T, grad_batch, levels == 2);
    *n_ops = (int64_t)prog.size();
    for (int64_t i = 0; i < (int64_t)prog.size() && i < max_ops; ++i) {
        const AdjOp &o = prog[(size_t)i];
        ops[3 * i] = o.op;
        ops[3 * i + 1] = o.a;
        ops[3 * i + 2] = o.b;
    }
    return STENCIL_OK;
}

int stencil_debug_bad_store(stencil_plan_t p, int64_t *index) {
    if (!p || !index) return STENCIL_EINVAL;
    if (!p->dbg) return STENCIL_EUNSUPPORTED;
    unsigned long long v = 0;
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(&v, p->dbg, sizeof(v), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e);
    *index = (int64_t)v - 1;
    return STENCIL_OK;
}

int stencil_pass_info(int kind, int dtype, int levels, int scheme, int variant, int64_t *info) {
    if (kind_radius(kind) < 0 || (dtype != STENCIL_F64 && dtype != STENCIL_F32) || !info || levels < 1)
        return STENCIL_EINVAL;
    bool ok = false;
    if (scheme == 3 && (variant == 0 || wf_tile(variant))) {
        const int tile = wf_tile(variant);
        ok = dtype == STENCIL_F32 ? wavefront_info_f32(kind, levels, tile, info)
                                  : wavefront_info_f64(kind, levels, tile, info);
    } else if (scheme == 4 && levels == 2 && dtype == STENCIL_F32) {
        ok = blk25_info_f32(kind, info);
    } else if (levels == 1 && variant >= 13 && variant <= 16) {
        ok = dtype == STENCIL_F32 ? plainv_info_f32(kind, variant, info) : plainv_info_f64(kind, variant, info);
    }
    return ok ? STENCIL_OK : STENCIL_EUNSUPPORTED;
}

int stencil_fma_peak(int dtype, void *stream, double *flops, double *sm_clock_hz) {
    if ((dtype != STENCIL_F64 && dtype != STENCIL_F32) || !flops || !sm_clock_hz) return STENCIL_EINVAL;
    cudaError_t e = run_fma_peak(dtype, (cudaStream_t)stream, flops, sm_clock_hz);
    return e == cudaSuccess ? STENCIL_OK : cuda_fail(e);
}

const char *stencil_strerror(int status) {
    switch (status) {
    case STENCIL_OK: return "ok";
    case STENCIL_EINVAL: return "invalid argument";
    case STENCIL_EUNSUPPORTED: return "unsupported by this build";
    case STENCIL_ENOMEM: return "device allocation failed";
    case STENCIL_ECUDA: return "CUDA error";
    case STENCIL_ETIMEOUT: return "a bounded device wait gave up";
    default: return "unknown status";
    }
}

int stencil_last_cuda_error(void) { return g_last_cuda_error; }

int stencil_wait_timeouts(int64_t *count) {
    if (!count) return STENCIL_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    *count = (int64_t)plainv_timeouts_f32() + (int64_t)plainv_timeouts_f64();
    return STENCIL_OK;
}

int stencil_check(stencil_plan_t p, void *stream) {
    if (!p) return STENCIL_EINVAL;
    cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
    if (e == cudaSuccess && p->grad_stream) e = cudaStreamSynchronize(p->grad_stream);
    if (e != cudaSuccess) return cuda_fail(e);
    const uint64_t now = (uint64_t)plainv_timeouts_f32() + plainv_timeouts_f64();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    const bool grew = now != p->timeouts_seen;
    p->timeouts_seen = now;
    return grew ? STENCIL_ETIMEOUT : STENCIL_OK;
}

}  // extern "C"
