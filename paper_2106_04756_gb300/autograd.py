"""torch.autograd.Function over the unrolled PDHG map.

The forward pass runs pdlp_unroll (T steps of Eq. (3) on the preconditioned
problem, step sizes from Algorithm 2 recorded and then held fixed, primal
weight fixed at its initial value) and returns (x_T, y_T) in the original
space; the backward pass is pdlp_grad, the hand-written adjoint of that map
(checkpointed every ckpt_every steps), giving the gradients with respect to
c, q and the nonzeros of K (CSR order).  Every step runs in the library's
CUDA kernels; this module only marshals tensors.

The library context lives as long as the autograd node that used it, so
backward may run more than once (retain_graph=True).  A caller that
evaluates the same LP repeatedly can pass its own `context` (created from
the same data) to skip the set-up of a new one per call; when that context
has run another unroll since this node's forward, the backward first
repeats this node's unroll (the map is deterministic, so the checkpoints it
rebuilds are the ones the forward saw).
"""
from __future__ import annotations

import torch

from . import Context


class UnrolledPDHG(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, q, k_val, row_ptr, col_idx, l, u, ineq, T, ckpt_every, options, context):
        n, m = c.numel(), q.numel()
        dev = c.device
        f64 = dict(dtype=torch.float64, device=dev)
        if context is None:
            lib_ctx = Context(row_ptr, col_idx, k_val.detach().contiguous(), c.detach().contiguous(),
                              q.detach().contiguous(), l, u, ineq, m, n, **(options or {}))
        else:
            lib_ctx = context
            if (lib_ctx.n, lib_ctx.m, lib_ctx.nnz) != (n, m, k_val.numel()):
                raise ValueError("context was created for an LP of other sizes")
        x = torch.empty(n, **f64)
        y = torch.empty(m, **f64)
        lib_ctx.pdlp_unroll(int(T), int(ckpt_every), x_out=x, y_out=y)
        ctx.lib_ctx = lib_ctx
        ctx.unroll = (int(T), int(ckpt_every), lib_ctx.unroll_generation)
        ctx.sizes = (n, m, k_val.numel(), dev)
        return x, y

    @staticmethod
    def backward(ctx, gx, gy):
        n, m, nnz, dev = ctx.sizes
        T, ckpt, gen = ctx.unroll
        f64 = dict(dtype=torch.float64, device=dev)
        lib_ctx = ctx.lib_ctx
        if lib_ctx.unroll_generation != gen:  # the shared context ran another unroll since
            lib_ctx.pdlp_unroll(T, ckpt)
            ctx.unroll = (T, ckpt, lib_ctx.unroll_generation)
        if gx is None:
            gx = torch.zeros(n, **f64)
        dc, dq, dk = torch.empty(n, **f64), torch.empty(m, **f64), torch.empty(nnz, **f64)
        lib_ctx.pdlp_grad(gx.contiguous(), None if gy is None else gy.contiguous(), dc=dc, dq=dq, dK=dk)
        return dc, dq, dk, None, None, None, None, None, None, None, None, None


def unrolled_pdhg(c, q, k_val, row_ptr, col_idx, l, u, ineq, T: int, ckpt_every: int = 50, context=None,
                  **options):
    """(x_T, y_T) of T unrolled PDHG steps, differentiable in c, q and k_val.

    All tensors on the same CUDA device: c, l, u float64[n]; q float64[m];
    k_val float64[nnz]; row_ptr int32[m+1]; col_idx int32[nnz]; ineq uint8[m]
    (1: row i is K_i x >= q_i).  options are pdlp_options fields.  context:
    an existing Context of this same LP to reuse (its data, not the tensors
    passed here, define the map), or None for a new one per call.
    """
    return UnrolledPDHG.apply(c, q, k_val, row_ptr, col_idx, l, u, ineq, T, ckpt_every, options, context)
