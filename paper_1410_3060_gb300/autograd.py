"""Receiver-misfit loss of a stencil time loop, differentiable with respect to
the initial field and the coefficient arrays.

    L(u0, W) = 0.5 * sum_{t=1..T} sum_{receiver plane} (u^t - d^t)^2,
    u^{-1} = u^0 = u0 (zero initial velocity for the wave kinds).

Forward: stencil_forward in segments of K steps (temporally blocked where
the library blocks the kind), keeping the state pair at every checkpoint
(every K steps) and the receiver trace; stencil_misfit gives the FP64 loss
and the residual.

Backward, segment by segment from the last: stencil_forward_states
recomputes the K states of the segment from its checkpoint, then
stencil_adjoint runs the transposed sweep backward over the segment,
injecting the residual on the receiver plane and accumulating the
coefficient gradients in FP64 (batched over steps).  The top segment starts
one level above T with a zero adjoint pair, so that lam^T = g^T is formed by
the library.  Finally dL/du0 = lam^0 - lam^1 (second-order kinds; the tied
u^{-1} contributes -lam^1) or lam^0 (first-order kinds), by stencil_axpby.

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
        return du0, dW.to(W.dtype), None, None


class MisfitRunner:
    """Checkpointed forward / adjoint driver for one plan.

    kind: a variable-coefficient kind (W25_VAR, J7_VAR, J25_VAR, W25_ALPHA);
    n = (nx, ny, nz); T steps; checkpoint every K steps; receivers on
    interior plane rcv_z; dtype st.F32 or st.F64; w: scalar weights of the
    kind (W25_ALPHA) or None.
    """

    def __init__(self, kind, n, T, K, rcv_z, dtype=st.F32, w=None, grad_batch=8, time_block=None):
        self.kind, self.n, self.T, self.K, self.rcv_z, self.w = kind, tuple(n), int(T), int(K), int(rcv_z), w
        self.plan = st.Plan(kind, *n, dtype)
        if time_block is not None:
            self.plan.set(st.OPT_TIME_BLOCK, time_block)
        self.plan.set(st.OPT_GRAD_BATCH, max(1, min(grad_batch, 16)))
        self.dtype = self.plan.torch_dtype()

    def close(self):
        self.plan.close()

    def __call__(self, u0, W, d):
        """Differentiable loss (0-dim FP64 tensor)."""
        return _MisfitFn.apply(u0, W, d, self)

    # -- forward: checkpoints, trace, loss
    def forward_pass(self, u0, W, d):
        T, K, (nx, ny, nz) = self.T, self.K, self.n
        dev = u0.device
        up, u = u0.detach().clone(), u0.detach().clone()
        trace = torch.empty((T, ny, nx), device=dev, dtype=self.dtype)
        ckpts = []
        t = 0
        while t < T:
            ckpts.append((t, up.clone(), u.clone()))
            k = min(K, T - t)
            self.plan.forward(up, u, self.w, W, k, trace=trace[t:t + k], rcv_z=self.rcv_z)
            t += k
        res = torch.zeros((T + 1, ny, nx), device=dev, dtype=self.dtype)  # res[i] = r^i, r^0 = 0
        loss = torch.zeros(1, device=dev, dtype=torch.float64)
        self.plan.misfit(trace, d, res[1:], loss)
        return loss[0], {"ckpts": ckpts, "res": res, "last": u}

    # -- backward: recompute + adjoint per segment
    def backward_pass(self, state, W, gloss):
        T, K, (nx, ny, nz) = self.T, self.K, self.n
        plan = self.plan
        res = state["res"]
        dev = res.device
        if not (isinstance(gloss, torch.Tensor) and gloss.numel() == 1):
            raise ValueError("scalar loss gradient expected")
        g = float(gloss.item())
        if g != 1.0:
            plan.axpby(g, res, 0.0, res, res)
        shape = plan.padded_shape
        lam_next = torch.zeros(shape, device=dev, dtype=self.dtype)
        lam = torch.zeros(shape, device=dev, dtype=self.dtype)
        grad = torch.zeros((st.NUM_ARRAYS[self.kind],) + shape, device=dev, dtype=torch.float64)
        bufs = [torch.zeros(shape, device=dev, dtype=self.dtype) for _ in range(K)]  # zero halo
        top = True
        for c, cp, cu in reversed(state["ckpts"]):
            k = min(K, T - c)
            # u^{c+1} .. u^{c+k} into bufs[0..k-1]
            plan.forward_states(cp, cu, self.w, W, bufs[:k])
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
        du0 = torch.empty(shape, device=dev, dtype=self.dtype)
        if st.SECOND_ORDER[self.kind]:
            plan.axpby(1.0, lam, -1.0, lam_next, du0)
        else:
            plan.axpby(1.0, lam, 0.0, lam, du0)
        return du0, grad


def misfit_loss(runner: MisfitRunner, u0, W, d):
    """Convenience: the differentiable receiver-misfit loss."""
    return runner(u0, W, d)
