"""Receiver-misfit loss of a stencil time loop, differentiable with respect to
the initial field and the coefficient arrays.

    L(u0, W) = 0.5 * sum_{t=1..T} sum_{receiver plane} (u^t - d^t)^2,
    u^{-1} = u^0 = u0 (zero initial velocity for the wave kinds).

Forward: stencil_forward in segments of K steps (temporally blocked where
the library blocks the kind), keeping the state pair at every checkpoint
(every K steps) and the receiver trace; stencil_misfit gives the FP64 loss
and the residual.  The last segment runs through stencil_forward_states,
so that its states are kept for the backward pass.

Backward, segment by segment from the last: stencil_forward_states
recomputes the K states of every earlier segment from its checkpoint (on a second
stream, one segment ahead, into the other of two state-buffer sets, so that
the recompute of segment i-1 overlaps the adjoint of segment i), then
stencil_adjoint runs the transposed sweep backward over the segment,
injecting the residual on the receiver plane and accumulating the
coefficient gradients in FP64 (batched over steps).  The top segment starts
one level above T with a zero adjoint pair, so that lam^T = g^T is formed by
the library.  Finally dL/du0 = lam^0 - lam^1 (second-order kinds; the tied
u^{-1} contributes -lam^1) or lam^0 (first-order kinds), by stencil_axpby.

Every forward pass gets its own set of checkpoint, trace, residual and loss
buffers from a pool of the runner (a new set is allocated only while more
forward passes are pending than the pool holds); the set returns to the
pool when the forward pass's state is dropped.  So several losses of one
runner may be built before a single backward() (their sum differentiates
correctly), and a forward pass under no_grad releases its set at once.

Every step of the computation runs in libstencil.so; torch provides memory
and the autograd plumbing.
"""
from __future__ import annotations

import torch

from . import stencil as st


class _MisfitFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, u0, W, d, runner):
        loss, state = runner.forward_pass(u0, W, d)
        ctx.runner = runner
        ctx.state = state
        ctx.save_for_backward(W)
        return loss

    @staticmethod
    def backward(ctx, gloss):
        (W,) = ctx.saved_tensors
        du0, dW = ctx.runner.backward_pass(ctx.state, W, gloss)
        ctx.state = None
        # the runner's gradient buffers are reused by its next backward pass
        return du0.clone(), dW.to(W.dtype, copy=True), None, None


class _ForwardState:
    """What one forward pass leaves for its backward pass: the checkpoints,
    the residual, and whether the last segment's states are still held.
    Owns one buffer set of the runner's pool and gives it back when dropped."""

    def __init__(self, runner, bufs):
        self._runner, self.bufs = runner, bufs
        self.ckpts, self.res, self.kept = [], bufs["res"], None

    def __del__(self):
        try:
            self._runner._pool.append(self.bufs)
        except Exception:
            pass


class MisfitRunner:
    """Checkpointed forward / adjoint driver for one plan.

    kind: a variable-coefficient kind (W25_VAR, J7_VAR, J25_VAR, W25_ALPHA);
    n = (nx, ny, nz); T steps; checkpoint every K steps; receivers on
    interior plane rcv_z; dtype st.F32 or st.F64; w: scalar weights of the
    kind (W25_ALPHA) or None.
    """

    def __init__(self, kind, n, T, K, rcv_z, dtype=st.F32, w=None, grad_batch=16, time_block=None,
                 device="cuda", overlap=True):
        self.kind, self.n, self.T, self.K, self.rcv_z, self.w = kind, tuple(n), int(T), int(K), int(rcv_z), w
        self.plan = st.Plan(kind, *n, dtype)
        if time_block is not None:
            self.plan.set(st.OPT_TIME_BLOCK, time_block)
        self.plan.set(st.OPT_GRAD_BATCH, max(1, min(grad_batch, 16)))
        self.dtype = self.plan.torch_dtype()
        # every buffer of a forward/backward pair is allocated once here (torch
        # owns the memory); the passes only clear them through the library
        nx, ny, nz = self.n
        shape = self.plan.padded_shape
        new = lambda *s_, dt=None: torch.empty(s_, device=device, dtype=dt or self.dtype)  # noqa: E731
        self._new = new
        self._pool = [self._new_forward_set()]
        self._state = (new(*shape), new(*shape))
        self._lam = (new(*shape), new(*shape))
        self._grad = new(st.NUM_ARRAYS[kind], *shape, dt=torch.float64)
        self.overlap = bool(overlap)
        self._sets = [[new(*shape) for _ in range(self.K)] for _ in range(2 if self.overlap else 1)]
        self._bufs = self._sets[0]
        self._du0 = new(*shape)
        for bs in self._sets:
            for b in bs:
                st.fill_zero(b)   # zero halos (only interiors are ever written)
        self._side = torch.cuda.Stream(device=device) if self.overlap else None
        self._kept = None
        self._res_scaled = None

    def _new_forward_set(self):
        """Checkpoints (state pair every K steps), trace, residual and loss of
        one forward pass."""
        nx, ny, nz = self.n
        shape = self.plan.padded_shape
        nck = (self.T + self.K - 1) // self.K
        return {"ckpt": [(self._new(*shape), self._new(*shape)) for _ in range(nck)],
                "trace": self._new(self.T, ny, nx), "res": self._new(self.T + 1, ny, nx),
                "loss": self._new(1, dt=torch.float64)}

    def close(self):
        self.plan.close()

    def __call__(self, u0, W, d):
        """Differentiable loss (0-dim FP64 tensor)."""
        return _MisfitFn.apply(u0, W, d, self)

    # -- forward: checkpoints, trace, loss
    def forward_pass(self, u0, W, d):
        T, K = self.T, self.K
        bufs = self._pool.pop() if self._pool else self._new_forward_set()
        state = _ForwardState(self, bufs)
        up, u = self._state
        u0d = u0.detach()
        up.copy_(u0d)
        u.copy_(u0d)
        trace = bufs["trace"]
        ckpts = state.ckpts
        t = 0
        nck = len(bufs["ckpt"])
        for i in range(nck):
            cp, cu = bufs["ckpt"][i]
            cp.copy_(up)
            cu.copy_(u)
            ckpts.append((t, cp, cu))
            k = min(K, T - t)
            if i == nck - 1:
                # the last segment's states are the first ones the backward
                # pass reads: they are kept (in the buffer set of the
                # backward's first segment) instead of being recomputed
                self.plan.forward_states(up, u, self.w, W, self._sets[0][:k], trace=trace[t:t + k],
                                         rcv_z=self.rcv_z)
            else:
                self.plan.forward(up, u, self.w, W, k, trace=trace[t:t + k], rcv_z=self.rcv_z)
            t += k
        res = bufs["res"]                    # res[i] = r^i, r^0 = 0
        st.fill_zero(res[0])
        self.plan.misfit(trace, d, res[1:], bufs["loss"])
        # the last segment's states sit in buffer set 0 until a backward
        # pass or a later forward pass reuses it
        self._kept = {"valid": True}
        state.kept = self._kept
        return bufs["loss"][0].clone(), state

    # -- backward: recompute + adjoint per segment
    def backward_pass(self, state, W, gloss):
        T, K, (nx, ny, nz) = self.T, self.K, self.n
        plan = self.plan
        res = state.res
        if not (isinstance(gloss, torch.Tensor) and gloss.numel() == 1):
            raise ValueError("scalar loss gradient expected")
        g = float(gloss.item())
        if g != 1.0:
            # scaled into the runner's scratch: the state's residual stays as
            # the forward pass left it (a later backward pass may reuse it)
            if self._res_scaled is None:
                self._res_scaled = torch.empty_like(res)
            plan.axpby(g, res, 0.0, res, self._res_scaled)
            res = self._res_scaled
        lam_next, lam = self._lam
        grad = self._grad
        for t_ in (lam_next, lam, grad):
            st.fill_zero(t_)
        segs = list(reversed(state.ckpts))
        main = torch.cuda.current_stream()
        nsets = len(self._sets)
        rec_ev, adj_ev = [None] * nsets, [None] * nsets
        # the forward pass left the last segment's states in buffer set 0,
        # valid until a backward pass (or a later forward pass) reuses the set
        kept = state.kept
        have_last = kept is not None and kept["valid"] and kept is self._kept
        # this pass rewrites the state-buffer sets: no forward pass's kept
        # states survive it
        if self._kept is not None:
            self._kept["valid"] = False

        def recompute(i, stream):
            # u^{c+1} .. u^{c+k} of segment i into buffer set i mod nsets
            c, cp, cu = segs[i]
            k = min(K, T - c)
            plan.forward_states(cp, cu, self.w, W, self._sets[i % nsets][:k], stream=stream)

        if self.overlap:
            self._side.wait_stream(main)          # checkpoints, residual and cleared buffers are ready
            if not have_last:
                with torch.cuda.stream(self._side):
                    recompute(0, self._side)
                    rec_ev[0] = self._side.record_event()
        top = True
        for i, (c, cp, cu) in enumerate(segs):
            k = min(K, T - c)
            if self.overlap:
                if i + 1 < len(segs):
                    # the next segment's states go into the set the adjoint of
                    # segment i - 1 read: wait for it, then recompute alongside
                    # this segment's adjoint
                    j = (i + 1) % nsets
                    with torch.cuda.stream(self._side):
                        if adj_ev[j] is not None:
                            self._side.wait_event(adj_ev[j])
                        recompute(i + 1, self._side)
                        rec_ev[j] = self._side.record_event()
                if rec_ev[i % nsets] is not None:
                    main.wait_event(rec_ev[i % nsets])
            elif not (i == 0 and have_last):
                recompute(i, main)
            bufs = self._sets[i % nsets]
            states = [cu] + bufs[:k - 1]
            if top:
                # start at level T+1 with (lam^{T+2}, lam^{T+1}) = 0: one extra step forms lam^T = g^T
                states = states + [bufs[k - 1]]
                plan.adjoint(lam_next, lam, self.w, W, k + 1, fwd_states=states, residual=res[c:T + 1],
                             rcv_z=self.rcv_z, grad=grad)
                top = False
            else:
                plan.adjoint(lam_next, lam, self.w, W, k, fwd_states=states, residual=res[c:c + k],
                             rcv_z=self.rcv_z, grad=grad)
            if self.overlap:
                adj_ev[i % nsets] = main.record_event()
        du0 = self._du0
        if st.SECOND_ORDER[self.kind]:
            plan.axpby(1.0, lam, -1.0, lam_next, du0)
        else:
            plan.axpby(1.0, lam, 0.0, lam, du0)
        return du0, grad


def misfit_loss(runner: MisfitRunner, u0, W, d):
    """Convenience: the differentiable receiver-misfit loss."""
    return runner(u0, W, d)
