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

using namespace stc;

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
std::vector<Op> build_program(int kind, int64_t T, int b) {
    std::vector<Op> ops;
    if (T <= 0) return ops;
    if (b < 1) b = 1;
    std::vector<int> L;
    const bool wave = kind_wave(kind);
    if (wave) {
        if (b == 1) {
            L.assign((size_t)T, 1);
        } else {
            for (int64_t i = 0; i < T / b; ++i) L.push_back(b);
            if (T % b) L.push_back((int)(T % b));
        }
        std::vector<bool> move(L.size());
        int nb = 0;
        for (size_t i = 0; i < L.size(); ++i) { move[i] = L[i] >= 2; nb += move[i]; }
        if (T == 1) {
            ops.push_back({0, 1, BUF_A, BUF_B, BUF_S1, BUF_S2});
            ops.push_back({1, 0, -1, BUF_S1, -1, BUF_A});
            ops.push_back({1, 0, -1, BUF_S2, -1, BUF_B});
            return ops;
        }
        if (nb % 2 == 1) {
            int last_plain = -1;
            for (size_t i = 0; i < L.size(); ++i) if (!move[i]) last_plain = (int)i;
            if (last_plain >= 0) {
                move[last_plain] = true;
            } else {
                // split the last blocked pass into (levels-1, 1), both moves
                const int v = L.back();
                L.back() = v - 1;
                L.push_back(1);
                move.push_back(true);
            }
            ++nb;
        }
        if (nb == 0 && T % 2 == 1) {
            int c = 0;
            for (int i = (int)L.size() - 1; i >= 0 && c < 2; --i) { move[i] = true; ++c; }
            nb = 2;
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
            const int64_t Tb = T - 1;
            for (int64_t i = 0; i < Tb / b; ++i) L.push_back(b);
            if (Tb % b) L.push_back((int)(Tb % b));
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
    double *partials;
    int npartials;
};

namespace {

int default_time_block(const stencil_plan_s *p) {
    if (p->dtype == STENCIL_F64) return 1;  // FP64 sweeps are bound by the FP64 pipe
    return blocked_default_levels(p->kind, p->dtype);
}

int effective_time_block(const stencil_plan_s *p) {
    int b = p->time_block > 0 ? p->time_block : default_time_block(p);
    if (b > 1 && !blocked_supported(p->kind, p->dtype, b)) b = 1;
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

template <typename T>
int run_program(stencil_plan_s *p, void *pair_p, void *pair_c, const stencil_coeffs_t *coeffs, int64_t nsteps,
                 cudaStream_t st, bool adjoint, void *trace, const void *inject, int64_t rcv_z,
                 const void *const *fwd_states, double *grad) {
    const int b = effective_time_block(p);
    const std::vector<Op> ops = build_program(p->kind, nsteps, b);
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
            SweepArgs<T> a;
            memset(&a, 0, sizeof(a));
            a.u_prev = (const T *)buf[o.in_p];
            a.u = (const T *)buf[o.in_c];
            a.out = (T *)buf[o.out_c];
            a.W = coeffs ? (const T *)coeffs->arrays : nullptr;
            a.s = s;
            a.g = p->g;
            a.rcv_z = (int)rcv_z;
            a.trace = (!adjoint && trace) ? (T *)trace + t * plane : nullptr;
            a.inject = (adjoint && inject) ? (const T *)inject + (nsteps - j) * plane : nullptr;
            cudaError_t e = launch_plain<T>(p->kind, adjoint, a, st, p->num_sms);
            if (e != cudaSuccess) return cuda_fail(e);
        } else {
            if (adjoint) return STENCIL_EUNSUPPORTED;
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
            cudaError_t e = launch_blocked<T>(p->kind, a, st, p->num_sms, p->scheme);
            if (e != cudaSuccess) return cuda_fail(e);
        }
        t += o.levels;
    }
    return STENCIL_OK;
}

void free_scratch(stencil_plan_s *p) {
    for (int i = 0; i < 2; ++i) {
        if (p->scratch[i]) cudaFree(p->scratch[i]);
        p->scratch[i] = nullptr;
    }
    if (p->partials) cudaFree(p->partials);
    p->partials = nullptr;
}

}  // namespace

extern "C" {

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
    *plan = p;
    return STENCIL_OK;
}

int stencil_plan_set(stencil_plan_t p, int option, int64_t value) {
    if (!p) return STENCIL_EINVAL;
    switch (option) {
    case STENCIL_OPT_TIME_BLOCK:
        if (value < 0 || value > 64) return STENCIL_EINVAL;
        if (value > 1 && !blocked_supported(p->kind, p->dtype, (int)value)) return STENCIL_EUNSUPPORTED;
        p->time_block = (int)value;
        return STENCIL_OK;
    case STENCIL_OPT_SCHEME:
        if (value < 0 || value > 2) return STENCIL_EINVAL;
        p->scheme = (int)value;
        return STENCIL_OK;
    default:
        return STENCIL_EINVAL;
    }
}

int stencil_plan_get(stencil_plan_t p, int option, int64_t *value) {
    if (!p || !value) return STENCIL_EINVAL;
    switch (option) {
    case STENCIL_OPT_TIME_BLOCK: *value = effective_time_block(p); return STENCIL_OK;
    case STENCIL_OPT_SCHEME: *value = p->scheme; return STENCIL_OK;
    case STENCIL_OPT_SCRATCH_BYTES:
        *value = (int64_t)((p->scratch[0] ? 2 * p->field_bytes : 0) + p->npartials * sizeof(double));
        return STENCIL_OK;
    default: return STENCIL_EINVAL;
    }
}

void stencil_plan_destroy(stencil_plan_t p) {
    if (!p) return;
    cudaDeviceSynchronize();
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
    if (p->dtype == STENCIL_F64)
        return run_program<double>(p, u_prev, u, coeffs, T, (cudaStream_t)stream, false, trace, nullptr,
                                   trace ? rcv_z : -1, nullptr, nullptr);
    return run_program<float>(p, u_prev, u, coeffs, T, (cudaStream_t)stream, false, trace, nullptr,
                              trace ? rcv_z : -1, nullptr, nullptr);
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
    // the adjoint runs plain passes (time block 1)
    const int saved = p->time_block;
    p->time_block = 1;
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

int stencil_schedule(int kind, int64_t T, int b, int32_t *ops, int64_t max_ops, int64_t *n_ops) {
    if (kind_radius(kind) < 0 || T < 0 || b < 1 || !n_ops || (max_ops > 0 && !ops)) return STENCIL_EINVAL;
    const std::vector<Op> prog = build_program(kind, T, b);
    *n_ops = (int64_t)prog.size();
    for (int64_t i = 0; i < (int64_t)prog.size() && i < max_ops; ++i) {
        const Op &o = prog[(size_t)i];
        const int32_t v[6] = {o.op, o.levels, o.in_p, o.in_c, o.out_p, o.out_c};
        memcpy(ops + 6 * i, v, sizeof(v));
    }
    return STENCIL_OK;
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
    default: return "unknown status";
    }
}

int stencil_last_cuda_error(void) { return g_last_cuda_error; }

}  // extern "C"
