/*
 * stencil.h -- C ABI of libstencil.so: temporally blocked 3D star-stencil
 * sweeps on NVIDIA GB300 (sm_103a).
 *
 * The operations follow the problem statement of Malas et al., "Multicore-
 * optimized wavefront diamond blocking for optimizing stencil updates"
 * (arXiv 1410.3060): a lattice Omega = {1..Nx} x {1..Ny} x {1..Nz}, x the
 * leading (unit-stride) dimension, stored as Omega[t][z][y][x] with two
 * time copies, swept T times by a Jacobi-style star-stencil update
 * (Sect. 3.1, Fig. 1).
 *
 * Layout (all arrays): halo-padded, dense, C order, extents
 * (nz+2R, ny+2R, nx+2R), x fastest.  The interior is padded index
 * R..R+n-1 in every axis; the halo of width R holds zero Dirichlet values,
 * must be zero on entry and is never written.  Coefficient stacks are
 * [k][nz+2R][ny+2R][nx+2R] in the plan's dtype; their halo values are not
 * read.  Device pointers must be 16-byte aligned.  "Interior plane z" below
 * means zero-based interior index z, padded plane z+R.
 *
 * Ownership and streams: the caller owns every array passed in.  A plan
 * owns only device scratch that it allocates in stencil_plan (and grows in
 * stencil_plan_set); stencil_forward / stencil_adjoint / stencil_misfit
 * allocate nothing.  Calls enqueue work on the given stream (a
 * cudaStream_t passed as void*, NULL = legacy default stream) and return
 * without synchronising.  One plan must not be used by two calls that
 * overlap in time (its scratch is shared).
 *
 * Errors: every int-returning call returns STENCIL_OK (0) or a negative
 * status; stencil_strerror names it.  STENCIL_ECUDA records the CUDA error,
 * readable through stencil_last_cuda_error.  Invalid arguments are
 * rejected on the host before any work is enqueued.
 */
#ifndef STENCIL_H
#define STENCIL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Operator kinds (paper Fig. 1).  Axis a: 0 = x, 1 = y, 2 = z.
 *  J7_CONST   Fig. 1b, radius 1:  u' = w1 u + w2 (x pair + y pair + z pair)
 *  J7_VAR     Fig. 1c, radius 1, 7 arrays at the updated point:
 *             u' = W0 u + W1 u[x-1] + W2 u[x+1] + W3 u[y-1] + W4 u[y+1]
 *                  + W5 u[z-1] + W6 u[z+1]
 *  W25_CONST  Fig. 1e with scalar alpha, radius 4, second order in time:
 *             u^{t+1} = 2u^t - u^{t-1} + alpha [w0 u^t + sum_r w_r (pairs
 *             at distance r along x, y and z)]; w0 is the 3D centre weight
 *  W25_VAR    radius 4, second order in time, 13 arrays with the Fig. 1d
 *             structure (index 0 centre, 3(r-1)+a+1 for the pair at
 *             distance r on axis a):
 *             u^{t+1} = 2u^t - u^{t-1} + W0 u^t + sum_{r,a} W_{3(r-1)+a+1} (pair)
 *  J25_VAR    Fig. 1d, radius 4, first order in time, 13 arrays:
 *             u' = W0 u + sum_{r,a} W_{3(r-1)+a+1} (pair)
 *  W25_ALPHA  Fig. 1e, radius 4, second order in time, domain-sized alpha:
 *             one array (alpha) and scalar weights w0..w4.                  */
enum stencil_kind {
    STENCIL_J7_CONST = 1,
    STENCIL_J7_VAR = 2,
    STENCIL_W25_CONST = 3,
    STENCIL_W25_VAR = 4,
    STENCIL_J25_VAR = 5,
    STENCIL_W25_ALPHA = 6
};

/* Storage and arithmetic precision of fields and coefficients. */
enum stencil_dtype { STENCIL_F64 = 0, STENCIL_F32 = 1 };

enum stencil_status {
    STENCIL_OK = 0,
    STENCIL_EINVAL = -1,       /* bad argument: see stencil_strerror        */
    STENCIL_EUNSUPPORTED = -2, /* valid request this build does not serve   */
    STENCIL_ENOMEM = -3,       /* device scratch allocation failed          */
    STENCIL_ECUDA = -4,        /* a CUDA call failed (stencil_last_cuda_error) */
    STENCIL_ETIMEOUT = -5      /* a bounded device wait gave up (stencil_check) */
};

/* Plan options (stencil_plan_set / stencil_plan_get). */
enum stencil_option {
    /* Time levels applied per pass over the lattice (the temporal block
       depth b).  0 = library default for the kind, dtype and scheme (3 for
       FP32 J7_CONST and 2 for FP32 J7_VAR on the register wavefront, 1 =
       plain sweeps otherwise), 1 = plain one-step-per-sweep kernel. */
    STENCIL_OPT_TIME_BLOCK = 1,
    /* Kernel family of a blocked pass: 0 = default (3 for FP32 7-point
       plans whose padded row length nx + 2 is even, 2 otherwise), 1 =
       shared-memory planes with overlapped tiles in x and y, 2 =
       shared-memory planes with diamond (split) tiles in y and overlapped x,
       3 = register wavefront with overlapped tiles (7-point kinds; FP32
       depths 1-4, FP64 depths 1-2; needs an even padded row length, else
       the plan runs plain passes), 4 = two-level pass of the 25-point
       kinds W25_VAR, J25_VAR and W25_CONST (FP32, depth 2, nx a multiple
       of 4): plane rings of both levels in shared memory, level-0 planes
       and u^{t-1} staged by TMA, the warps split by level. */
    STENCIL_OPT_SCHEME = 2,
    /* Read-only: bytes of device scratch the plan holds. */
    STENCIL_OPT_SCRATCH_BYTES = 3,
    /* Adjoint steps whose coefficient-gradient terms are summed in FP64
       registers before one read-modify-write of the gradient arrays
       (1..16, default 1).  G > 1 makes the plan hold 2G + 2 state fields of
       scratch in which stencil_adjoint keeps the adjoint levels of two
       batches: the gradient of one batch runs on a plan-owned stream while
       the sweeps of the next batch run on the caller's stream (the call
       still returns with all of its work ordered on the caller's stream). */
    STENCIL_OPT_GRAD_BATCH = 4,
    /* Tile variant of the plain forward sweep (the tuning parameter of the
       one-level kernel): 0 = measured default for the kind and dtype,
       1..4, 6, 7 = asynchronously staged tiles of 32x8, 32x16, 32x16 (4 rows
       per thread), 64x8, 64x16 and 128x8 columns, 5 = register-staged 2.5D
       kernel, 8 and 9 = 32x8 and 32x16 tiles with the per-point inputs
       (coefficients, u^{t-1}) staged asynchronously as well, 10..12 =
       register wavefront tiles of 64x32 (4 rows per thread), 64x32 (2 rows
       per thread) and 64x64 points (7-point kinds; the same tiles serve the
       blocked passes of scheme 3), 13 and 14 = vectorised sweep of the
       25-point kinds with 16-byte vectors along x, 8 and 16 rows per CTA
       (4 rows for the 13-array kinds; needs nx a multiple of 4 in FP32, of
       2 in FP64), 15 and 16 = the same tiles staged by TMA (one tensor copy
       per plane tile, mbarrier completion; the adjoint of W25_VAR and
       J25_VAR then stages every coefficient tile by TMA as well), 17 =
       FP32 register wavefront tile of 128x32 points, 4 points per thread
       row and 2 rows per thread (128x16 at depth 4; an FP64 plan rejects
       it with EUNSUPPORTED).  A
       variant a kind or geometry cannot use runs the default streaming
       tile.  The
       default is the measured best: 12 / 11 for FP32 J7_CONST / J7_VAR (the
       one-level passes of a default J7_CONST plan run 11), 15
       for FP32 W25_CONST, 16 for FP32 W25_ALPHA and for W25_VAR and
       J25_VAR, else a streaming tile. */
    STENCIL_OPT_VARIANT = 5,
    /* 1: stencil_forward captures its pass program (every launch and copy of
       the T steps) into a CUDA graph the first time it sees an argument set
       (state pair, coefficients, T, trace, rcv_z and the tuning options) and
       replays that graph on the caller's stream while the arguments stay
       the same; a new argument set or any stencil_plan_set replaces the
       graph.  Capture runs on a plan-owned stream, so the caller's stream
       may be the legacy default stream.  0 (default): direct launches. */
    STENCIL_OPT_GRAPH = 6,
    /* Polls of the bounded mbarrier waits of the TMA-staged sweeps (tile
       variants 15 and 16) before a wait gives up: 0 = default (2^22, far
       longer than any copy takes; each poll may suspend the thread for a
       hardware-defined time).  A CTA whose wait gives up stops sweeping,
       waits (bounded) for its copies in flight and returns; its part of the
       result is then wrong and stencil_check reports STENCIL_ETIMEOUT. */
    STENCIL_OPT_WAIT_LIMIT = 7,
    /* Test hook for the give-up path of the bounded waits: v >= 0 makes the
       first CTA (block 0, 0, 0) of every TMA-staged sweep of this plan skip
       issuing the copies of interior plane v (the first CTA's first z chunk
       then waits for a copy that never comes, gives up and returns; no copy
       is left in flight).  -1 = off (default).  Only for tests of the
       ETIMEOUT path, together with a small STENCIL_OPT_WAIT_LIMIT. */
    STENCIL_OPT_TEST_SKIP_COPY = 8,
    /* Time levels per pass of stencil_adjoint (Sect. 4.1 wavefront applied
       to the transposed sweep): 1 = one level per pass, 2 = passes of two
       levels for the 7-point kinds (the register wavefront's adjoint) and,
       in FP32, the 13-array kinds W25_VAR and J25_VAR (the two-level pass's
       adjoint, nx a multiple of 4); each pass reads lam^{t+1} (and
       lam^{t+2}) and the coefficients once and writes lam^t and lam^{t-1};
       EUNSUPPORTED for other kinds or geometries the pass does not serve.  With a gradient, levels are paired only
       inside a gradient batch (STENCIL_OPT_GRAD_BATCH >= 2); with batch 1
       every pass is one level.  0 = default: 2 for the FP32 7-point kinds
       (measured at 512^3: 7-point variable 259 vs 129 GLUP/s, constant 789
       vs 584), else 1 (FP64 is bound by the FP64 pipe either way; the
       13-array kinds' pass measures 37-39 vs 91-94 GLUP/s).  Passes run
       the plan's register wavefront tile (variants 10-12), else the 64x32
       tile of 2 rows per thread (variable kind) or the 64x64 tile
       (constant kind).  Reading it gives the depth the adjoint runs. */
    STENCIL_OPT_ADJ_TIME_BLOCK = 9
};

typedef struct stencil_plan_s *stencil_plan_t;

/* Coefficients of one call.
 *  w:      host array of nw FP64 scalars, for the kinds that take them:
 *          J7_CONST {w1, w2}; W25_CONST {alpha, w0, w1, w2, w3, w4};
 *          W25_ALPHA {w0, w1, w2, w3, w4}; NULL / 0 otherwise.  Copied at
 *          the call; need not outlive it.
 *  arrays: device coefficient stack in the plan's dtype, k arrays of the
 *          padded extent: J7_VAR k = 7, W25_VAR and J25_VAR k = 13,
 *          W25_ALPHA k = 1 (alpha); NULL for the constant kinds.  For the
 *          adjoint its halo entries must be finite.                        */
typedef struct {
    const double *w;
    int32_t nw;
    const void *arrays;
} stencil_coeffs_t;

/* Create a plan for one operator on an nx x ny x nz interior
 * (Sect. 3.1 problem statement).  radius must equal the kind's radius (1
 * or 4); every n must be >= 1.  Allocates the plan's device scratch on the
 * current device.  Returns EINVAL for a bad kind/radius/dtype/size, ENOMEM
 * if scratch cannot be allocated. */
int stencil_plan(stencil_plan_t *plan, int kind, int64_t nx, int64_t ny, int64_t nz,
                 int radius, int dtype);

/* Set / read a plan option (enum stencil_option).  Setting may reallocate
 * the plan's scratch; it must not race with work enqueued on the plan. */
int stencil_plan_set(stencil_plan_t plan, int option, int64_t value);
int stencil_plan_get(stencil_plan_t plan, int option, int64_t *value);

/* Release the plan and its scratch (synchronises the device first). */
void stencil_plan_destroy(stencil_plan_t plan);

/* Advance the state T time steps (Sect. 3.1: the sweep repeated T times;
 * temporally blocked per Sect. 4: several time levels per pass).
 *  u_prev, u: device state pair.  On entry (u_prev, u) = (u^{-1}, u^0);
 *             first-order kinds ignore u_prev's entry contents.  On return
 *             (u_prev, u) = (u^{T-1}, u^T).  T = 0 leaves both untouched.
 *             u_prev and u must be distinct, non-overlapping arrays.
 *  trace:     NULL, or device [T][ny][nx] (plan dtype) receiving
 *             trace[t] = u^{t+1} on interior plane rcv_z, 0 <= rcv_z < nz.
 * Results match the naive sweep of Fig. 1 up to rounding order. */
int stencil_forward(stencil_plan_t plan, void *u_prev, void *u, const stencil_coeffs_t *coeffs,
                    int64_t T, void *stream, void *trace, int64_t rcv_z);

/* Forward T steps storing every state (the recompute pass of checkpointed
 * differentiation): states is a host array of T device pointers, states[t]
 * receives u^{t+1}.  u_prev, u hold (u^{-1}, u^0) and are only read.
 * trace / rcv_z as in stencil_forward.  The state arrays must be distinct
 * from each other and from the inputs, and their halos must be zero (only
 * interiors are written).  Plain one-level sweeps, except for the 7-point
 * kinds on a plan whose passes run the register wavefront at depth >= 2
 * (the FP32 default): there one depth-2 pass writes two consecutive
 * states. */
int stencil_forward_states(stencil_plan_t plan, const void *u_prev, const void *u,
                           const stencil_coeffs_t *coeffs, int64_t T, void *const *states,
                           void *stream, void *trace, int64_t rcv_z);

/* T steps of the adjoint (transposed) sweep, backward in time (one or two
 * levels per pass, STENCIL_OPT_ADJ_TIME_BLOCK), for a loss
 * L = sum_n l_n(u^n) with explicit partials g^n = P^T r^n injected on
 * receiver plane rcv_z.  With A the spatial operator and A^T its transpose
 * ((A^T y)(q) = sum_k A_k(q - o_k) y(q - o_k) over interior source points):
 *   first-order kinds:  lam^n = g^n + A^T lam^{n+1}
 *   second-order kinds: lam^n = g^n + 2 lam^{n+1} + A^T lam^{n+1} - lam^{n+2}
 *  lam_next, lam: device pair.  On entry (lam^{m+1}, lam^m), g^m already in
 *             lam^m; on return (lam^{m-T+1}, lam^{m-T}).
 *  fwd_states: host array of T device pointers, fwd_states[i] = u^{m-T+i};
 *             required when grad is non-NULL, otherwise ignored.
 *  residual:  NULL, or device [T][ny][nx] (plan dtype), residual[i] = r^{m-T+i}
 *             added to lam^{m-T+i} on plane rcv_z.
 *  grad:      NULL, or device FP64 [k][nz+2R][ny+2R][nx+2R] (variable-
 *             coefficient kinds only): accumulates, interior entries only,
 *             dL/dA_k(x) += sum_n lam^{n+1}(x) d(A u^n)(x)/dA_k(x).
 * The adjoint of the constant-coefficient kinds returns EUNSUPPORTED when
 * grad is non-NULL. */
int stencil_adjoint(stencil_plan_t plan, void *lam_next, void *lam, const stencil_coeffs_t *coeffs,
                    int64_t T, void *stream, const void *const *fwd_states, const void *residual,
                    int64_t rcv_z, double *grad);

/* out[i] = alpha * x[i] + beta * y[i] for n elements of the plan's dtype
 * (the gradient with respect to a tied initial state, dL/du0 = lam^0 -
 * lam^1 for second-order kinds with u^{-1} = u^0, and the scaling of a
 * residual by an incoming loss gradient).  out may alias x or y. */
int stencil_axpby(stencil_plan_t plan, int64_t n, double alpha, const void *x, double beta,
                  const void *y, void *out, void *stream);

/* Set `bytes` bytes of device memory to zero on `stream` (asynchronous
 * cudaMemsetAsync): clears the caller's state, adjoint and gradient arrays
 * (whose halos must be zero) without leaving the library. */
int stencil_fill_zero(void *ptr, int64_t bytes, void *stream);

/* Receiver misfit of T traces: residual = trace - d (plan dtype, may alias
 * neither input unless equal to trace), and *loss (device FP64) =
 * 0.5 * sum (trace - d)^2 accumulated in FP64 in a fixed order
 * (deterministic).  trace, d, residual: device [T][ny][nx]. */
int stencil_misfit(stencil_plan_t plan, const void *trace, const void *d, int64_t T, void *residual,
                   double *loss, void *stream);

/* Receiver misfit that allocates nothing: the same result as
 * stencil_misfit (residual = trace - d, *loss = 0.5 * sum (trace - d)^2 in
 * FP64, fixed summation order), without a plan.  The paper has no
 * counterpart; this entry exists for callers that cannot allocate device
 * memory themselves -- code embedded in an application whose device memory
 * is owned by its own allocator (raw cudaMalloc/cudaFree are not allowed or
 * would fragment its pool), or latency-critical loops where a device
 * allocation, which may synchronise the device, is not acceptable.
 *  dtype: STENCIL_F64 or STENCIL_F32; trace, d, residual: device arrays of
 *         n elements of that type (caller-owned); loss: device FP64.
 *  n must be <= STENCIL_MISFIT_STATIC_MAX_ELEMS, else STENCIL_EINVAL (no
 *  work is enqueued).
 * Scratch: the FP64 partial sums live in a static device array of the
 * library (64 KiB, one partial per 2048 elements, at most 8192), which every
 * GPU that loads the library holds until the process exits.  A call looks up
 * that array's device address (cudaGetSymbolAddress, with the device
 * current) unless its stream is being captured; inside a capture it uses the
 * address found by an earlier call on that device, so make one call on each
 * device before any stream capture (a capture without one fails with
 * STENCIL_ECUDA).
 * All calls share the array: calls that may overlap on the GPU (different
 * streams, or other threads) race and must be serialised by the caller.
 * Every entry a call reads is written by the same call, so nothing carries
 * over between calls.  Calls no cudaMalloc / cudaFree. */
#define STENCIL_MISFIT_STATIC_MAX_ELEMS ((int64_t)8192 * 2048)
int stencil_misfit_static(int dtype, const void *trace, const void *d, int64_t n, void *residual,
                          double *loss, void *stream);

/* Host-only: the program of passes and copies that stencil_forward (and,
 * with the same rules, stencil_adjoint) runs for T steps of `kind` in
 * `dtype` with temporal block depth b (b >= 1; 1 = plain sweeps; a depth
 * the kernels do not provide falls back to 1, and remainders use the
 * provided depths).  Each op is 6 int32:
 *   {op, levels, in_prev, in_cur, out_prev, out_cur}
 * op 0 = pass over the lattice applying `levels` time levels, op 1 = copy
 * of buffer in_cur to out_cur.  Buffer ids: 0 = the caller's u_prev,
 * 1 = the caller's u, 2 and 3 = plan scratch fields, -1 = not used.  A pass
 * reads (in_prev, in_cur) = (u^{t-1}, u^t) and writes u^{t+levels} to
 * out_cur and, when out_prev >= 0, u^{t+levels-1} to out_prev; out_cur ==
 * in_prev marks an in-place second-order update.  Writes at most max_ops
 * ops and the total count to *n_ops.  Performs no CUDA call. */
int stencil_schedule(int kind, int dtype, int64_t T, int b, int32_t *ops, int64_t max_ops, int64_t *n_ops);

/* The host program stencil_adjoint runs for T steps with a gradient in
 * batches of grad_batch steps (1..16, STENCIL_OPT_GRAD_BATCH >= 2) and
 * `levels` (1 or 2) levels per pass where the plan allows them (the
 * adjoint form of the time-loop driver, Sect. 3.1 recursion run backward):
 * ops receives up to max_ops triples (op, a, b) in issue order, *n_ops the
 * total count --
 *   (0, b, 0)  the caller's stream waits for gradient batch b - 2 before
 *              batch b's first sweep (the sweeps of batch b overwrite the
 *              ring slots that batch reads);
 *   (1, j, n)  the sweep of steps j .. j+n-1 (n = 1 or 2; step j produces
 *              lam^{m-j} into ring slot (j-1) mod (2 grad_batch + 2));
 *   (2, b, k)  gradient batch b of k steps on the plan's gradient stream.
 * Host-only (no CUDA call); EINVAL for a bad argument. */
int stencil_adjoint_schedule(int64_t T, int grad_batch, int levels, int64_t *ops, int64_t max_ops,
                             int64_t *n_ops);

/* Debug builds (compiled with -DSTENCIL_DEBUG) check every store of a
 * sweep's result: a store whose target is not an interior point of the
 * padded array (a sweep never writes the halo or outside the array) is
 * skipped and its linear element index recorded -- the kernels record and
 * skip, they never trap.  Into *index: the first such index recorded by the
 * plan's sweeps since its creation, or -1 if none.  Synchronises the
 * device.  STENCIL_EUNSUPPORTED in the normal build. */
int stencil_debug_bad_store(stencil_plan_t plan, int64_t *index);

/* Host-only: the on-chip resources of one pass-kernel configuration -- the
 * GPU counterpart of the cache block of a wavefront tile (Sect. 5.3): what
 * one CTA keeps in shared memory while it marches through z.  Into
 * info[0..5]: dynamic shared memory per CTA (bytes), threads per CTA, the x
 * and y extent of the points a CTA computes per plane (owned points plus the
 * overlapped halo of a blocked pass), and the x and y extent of the points it
 * owns.  Served for the register wavefront (scheme 3, variant 0 = its
 * default tile or 10-12, every depth it supports: 1-4 FP32, 1-2 FP64, 7-point
 * kinds), the two-level pass of the 25-point kinds (scheme 4: W25_VAR,
 * J25_VAR, W25_CONST; levels 2, FP32) and the vectorised one-level sweep (levels 1, variants 13-16);
 * STENCIL_EUNSUPPORTED for other families, STENCIL_EINVAL for a bad
 * argument.  Performs no CUDA call. */
int stencil_pass_info(int kind, int dtype, int levels, int scheme, int variant, int64_t *info);

/* Measure the device's FP64 (dtype STENCIL_F64) or FP32 fused multiply-add
 * throughput with independent FMA chains on every SM: *flops = flops per
 * second (FMA = 2), *sm_clock_hz = SM clock seen by the kernel's cycle
 * counter.  Synchronises the stream; used as the roofline denominator of
 * ALU-bound kernels. */
int stencil_fma_peak(int dtype, void *stream, double *flops, double *sm_clock_hz);

/* Name of a status code. */
const char *stencil_strerror(int status);

/* The last CUDA error code recorded by a call that returned STENCIL_ECUDA
 * in this thread (cudaError_t as int), or 0. */
int stencil_last_cuda_error(void);

/* Number of CTAs of the TMA-staged sweeps whose bounded wait for a plane
 * copy gave up since the library was loaded, on the current device, into
 * *count (0 on a healthy run).  Such a CTA leaves its sweep with every
 * other thread of the CTA at the barrier after the wait, waits (bounded)
 * for the copies it still has in flight and returns, so the kernel ends
 * instead of hanging; its part of the result is wrong.  Synchronises the
 * device. */
int stencil_wait_timeouts(int64_t *count);

/* Wait for the work enqueued on `stream` (and on the plan's own gradient
 * stream) to finish and report its status: STENCIL_ETIMEOUT if any bounded
 * device wait of the library gave up since the plan's previous
 * stencil_check (or its creation) -- the results of the calls in between
 * are then invalid --, STENCIL_ECUDA if a CUDA error was reported, else
 * STENCIL_OK.  The device counters are shared by all plans of the process:
 * a timeout in another plan's work in that interval is reported too. */
int stencil_check(stencil_plan_t plan, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* STENCIL_H */
