"""torch.autograd.Function over the sampler's action (argument marshalling only).

forward: A(X, p) = A_o + A_f (FP64 sums) by pimc_action_dev;
backward: dA/dX, dA/dp by the reverse-mode adjoint through the RK4 map with the
stages recomputed (pimc_grad_dev), scaled by the incoming gradient.  Both run
on the tensors' CUDA stream; X is (D, M+1) float64, p is (Np,) float64, both
contiguous on the GPU.
"""
from __future__ import annotations

import torch

from . import pimc as _pimc


class PathAction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, X, p, sampler):
        if X.dtype != torch.float64 or p.dtype != torch.float64 or not X.is_cuda or not p.is_cuda:
            raise TypeError("PathAction expects float64 CUDA tensors")
        X = X.contiguous()
        p = p.contiguous()
        if X.shape != (sampler.D, sampler.M + 1) or p.shape != (sampler.Np,):
            raise ValueError("X must be (D, M+1) and p (Np,)")
        out = torch.empty(3, dtype=torch.float64, device=X.device)
        stream = torch.cuda.current_stream(X.device).cuda_stream
        sampler.action_dev(X.data_ptr(), p.data_ptr(), out.data_ptr(), stream)
        ctx.save_for_backward(X, p)
        ctx.sampler = sampler
        return out[0]

    @staticmethod
    def backward(ctx, grad_out):
        X, p = ctx.saved_tensors
        gX = torch.empty_like(X)
        gp = torch.empty_like(p)
        stream = torch.cuda.current_stream(X.device).cuda_stream
        ctx.sampler.grad_dev(X.data_ptr(), p.data_ptr(), 1.0, gX.data_ptr(), gp.data_ptr(), stream)
        return grad_out * gX, grad_out * gp, None


def path_action(X: torch.Tensor, p: torch.Tensor, sampler: "_pimc.Sampler") -> torch.Tensor:
    """Differentiable action of the path X and parameters p for `sampler`'s data."""
    return PathAction.apply(X, p, sampler)
