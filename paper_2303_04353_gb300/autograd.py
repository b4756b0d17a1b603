"""Differentiable FP64x2 GEMM.

``DDMatmul`` wraps the cascade as a ``torch.autograd.Function`` whose
backward is hand-written: dA = dC B^T and dB = A^T dC, each computed by the
same cascade kernels (``ddgemm_backward`` in the C ABI).  The paper has no
backward pass; this is the chain rule applied to its product.

Convention: an FP64x2 tensor is the pair (hi, lo) and its value is hi + lo.
Its cotangent is FP64x2 too and is carried by the pair of gradients:
the cotangent of C is grad(c_hi) + grad(c_lo), and after backward
a_hi.grad + a_lo.grad is dL/dA (likewise for B).  For a loss L = sum(W * C)
with W = (w_hi, w_lo), call ``torch.autograd.backward((c_hi, c_lo),
(w_hi, w_lo))``."""
from __future__ import annotations

import torch

from . import ops


class DDMatmul(torch.autograd.Function):
    @staticmethod
    def forward(ctx, a_hi, a_lo, b_hi, b_lo, variant=0):
        c_hi, c_lo = ops.ddgemm(a_hi, a_lo, b_hi, b_lo, variant=variant)
        ctx.save_for_backward(a_hi, a_lo, b_hi, b_lo)
        ctx.variant = variant
        return c_hi, c_lo

    @staticmethod
    def backward(ctx, g_hi, g_lo):
        a_hi, a_lo, b_hi, b_lo = ctx.saved_tensors
        ref = g_hi if g_hi is not None else g_lo
        if ref is None:
            return None, None, None, None, None
        g_hi = torch.zeros_like(ref) if g_hi is None else g_hi.contiguous()
        g_lo = torch.zeros_like(ref) if g_lo is None else g_lo.contiguous()
        da_hi, da_lo, db_hi, db_lo = ops.ddgemm_backward(a_hi, a_lo, b_hi, b_lo, g_hi, g_lo,
                                                         variant=ctx.variant)
        return da_hi, da_lo, db_hi, db_lo, None


def ddmatmul(a_hi, a_lo, b_hi, b_lo, variant=0):
    """C = A B in FP64x2 (differentiable); returns (c_hi, c_lo).  variant:
    0 the FP64 form (default), 1 the INT8 form on mma.sync, 4 the INT8 form
    on the tcgen05 tensor cores (seven-bit pieces), 5 the same with
    eight-bit pieces; forward and backward use the same form."""
    return DDMatmul.apply(a_hi, a_lo, b_hi, b_lo, variant)
