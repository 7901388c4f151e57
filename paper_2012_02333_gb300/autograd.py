"""torch.autograd wrappers of the reconstruction and of its adjoint.

Reconstruct.apply(cc, algo, *tensors) -> p (2^n probabilities); its backward
calls cutqc_reconstruct_backward with the incoming gradient as G.

MaxCutExpectation.apply(cc, edges, *tensors) -> L = sum_x C(x) p(x), the
expected cut size under the reconstructed distribution, computed together
with dL/dT_c by the library's MaxCut adjoint (no 2^n array is formed).
"""
from __future__ import annotations

import torch

from . import cutqc


class Reconstruct(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cc, algo, *tensors):
        ts = [t.contiguous() for t in tensors]
        out, _ = cutqc.reconstruct_fd(cc, ts, algo=algo, with_sum=False)
        ctx.cc = cc
        ctx.save_for_backward(*ts)
        return out

    @staticmethod
    def backward(ctx, grad_p):
        ts = ctx.saved_tensors
        problem = cutqc.Problem.from_cut(ctx.cc, list(ts))
        grads = [torch.empty_like(t) for t in ts]
        cutqc.cutqc_reconstruct_backward(problem, grads, grad_out=grad_p.contiguous().to(ts[0].dtype))
        return (None, None, *grads)


class MaxCutExpectation(torch.autograd.Function):
    @staticmethod
    def forward(ctx, cc, edges, *tensors):
        ts = [t.contiguous() for t in tensors]
        problem = cutqc.Problem.from_cut(cc, ts)
        grads = [torch.empty_like(t) for t in ts]
        loss = torch.empty(1, dtype=torch.float64, device=ts[0].device)
        cutqc.cutqc_reconstruct_backward(problem, grads, edges=edges, loss_value=loss)
        ctx.grads = grads
        return loss[0]

    @staticmethod
    def backward(ctx, g):
        return (None, None, *[gr * g.to(gr.dtype) for gr in ctx.grads])
