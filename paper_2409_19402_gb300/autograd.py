"""Differentiable projected product C = A *Q B (Def. 3.1) for PyTorch autograd.

Forward and backward both run through the C ABI (pprod / pprod_backward): the
backward recomputes the transform-domain tensors A-hat, B-hat, C-hat instead
of storing them, and returns for Q the gradient projected on the tangent space
of the Stiefel manifold St_{n,p} at Q (set ``stiefel=False`` for the Euclidean
gradient).  Inputs of lower precision (e.g. bfloat16) are computed in FP32 and
the results cast back to the input dtype.
"""
from __future__ import annotations

import torch

from . import binding


class _QProd(torch.autograd.Function):
    @staticmethod
    def forward(ctx, A, B, Q, stiefel):
        dt = A.dtype
        A32, B32, Q32 = (x.detach().float().contiguous() for x in (A, B, Q))
        C = binding.pprod(A32, B32, Q32)
        ctx.save_for_backward(A32, B32, Q32)
        ctx.stiefel = bool(stiefel)
        ctx.dtypes = (A.dtype, B.dtype, Q.dtype)
        return C.to(dt)

    @staticmethod
    def backward(ctx, G):
        A32, B32, Q32 = ctx.saved_tensors
        dA, dB, dQ, dQE = binding.pprod_backward(A32, B32, Q32, G.float().contiguous(),
                                                 want_euclid=not ctx.stiefel)
        gq = dQ if ctx.stiefel else dQE
        ta, tb, tq = ctx.dtypes
        return dA.to(ta), dB.to(tb), gq.to(tq), None


def qprod(A: torch.Tensor, B: torch.Tensor, Q: torch.Tensor, stiefel: bool = True) -> torch.Tensor:
    """C = A *Q B with A (n, n1, m), B (n, m, n2), Q (n, p) CUDA tensors."""
    return _QProd.apply(A, B, Q, stiefel)
