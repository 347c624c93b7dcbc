"""torch.autograd.Function over the hand-written loss and adjoint kernels.

``starred_loss(params, problem)`` returns the loss as a 0-d float64 CUDA tensor;
its backward returns the gradient computed by the library's adjoint kernels in
the same call (no intermediates are kept per epoch: the supersampled images are
recomputed inside the kernels).
"""
from __future__ import annotations

import torch


class StarredLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params: torch.Tensor, problem) -> torch.Tensor:
        loss, grad = problem.loss_and_grad(params.detach().contiguous(), sync=False)
        ctx.save_for_backward(grad)
        return loss

    @staticmethod
    def backward(ctx, grad_out: torch.Tensor):
        (grad,) = ctx.saved_tensors
        return (grad_out.to(grad.dtype) * grad, None)


def starred_loss(params: torch.Tensor, problem) -> torch.Tensor:
    return StarredLoss.apply(params, problem)
