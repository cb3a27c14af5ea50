"""Differentiable masked product C = M .* (A B) on plus-times fp32.

The loss l(C) reaches A and B through C's values only.  With G = dl/dC stored
on C's pattern, dA = pattern(A) .* (G B^T) and dB = pattern(B) .* (A^T G);
both are masked products run by the library's own accumulators
(``msgemm_backward_planned``).  Patterns are fixed; gradients flow to the
value arrays of A and B, and the transposed patterns the backward needs are
built once per (A, B) pattern pair and handle.
"""
from __future__ import annotations

import torch

from ._lib import BackwardPlan, DeviceCsr, Handle, msgemm_backward, msgemm_run


def backward_plan(handle: Handle, A: DeviceCsr, B: DeviceCsr) -> BackwardPlan:
    """The backward plan of (A, B) on this handle, made on first use and kept
    on A (patterns are fixed; only values change between steps)."""
    plans = A.__dict__.setdefault("_backward_plans", {})
    key = (id(handle), id(B))
    plan = plans.get(key)
    if plan is None or plan.p is None:
        plan = BackwardPlan(handle, A, B)
        plans[key] = plan
    return plan


class MaskedSpGEMM(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_vals: torch.Tensor, b_vals: torch.Tensor, M: DeviceCsr, A: DeviceCsr, B: DeviceCsr,
                handle: Handle):
        Ax = DeviceCsr(A.nrows, A.ncols, A.rowptr, A.colidx, a_vals.detach().contiguous())
        Bx = DeviceCsr(B.nrows, B.ncols, B.rowptr, B.colidx, b_vals.detach().contiguous())
        res = msgemm_run(handle, M, Ax, Bx, "plus_times_f32", False)
        c = res.trimmed()
        ctx.save_for_backward(a_vals, b_vals)
        ctx.pattern = (c.rowptr, c.colidx)
        ctx.mats = (M, A, B, handle)
        ctx.mark_non_differentiable(c.rowptr, c.colidx)
        return c.values, c.rowptr, c.colidx

    @staticmethod
    def backward(ctx, g_vals, _g_rp=None, _g_ci=None):
        a_vals, b_vals = ctx.saved_tensors
        M, A, B, handle = ctx.mats
        rp, ci = ctx.pattern
        G = DeviceCsr(M.nrows, M.ncols, rp, ci, g_vals.contiguous().float())
        Ax = DeviceCsr(A.nrows, A.ncols, A.rowptr, A.colidx, a_vals.detach().contiguous())
        Bx = DeviceCsr(B.nrows, B.ncols, B.rowptr, B.colidx, b_vals.detach().contiguous())
        dA, dB = msgemm_backward(handle, Ax, Bx, G, ctx.needs_input_grad[0], ctx.needs_input_grad[1],
                                 plan=backward_plan(handle, A, B))
        return dA, dB, None, None, None, None


def masked_spgemm_autograd(a_vals, b_vals, M: DeviceCsr, A: DeviceCsr, B: DeviceCsr, handle: Handle):
    """Returns (C values, C rowptr, C colidx); C values carry gradients to
    a_vals and b_vals."""
    return MaskedSpGEMM.apply(a_vals, b_vals, M, A, B, handle)
