"""torch.autograd.Function wrappers of the library's hand-written backward.

``OneHotLoss``   L(g(W)) of eq. 7 at the one-hot population S = g(W) with the
                 straight-through gradient of eq. 12-13 as its backward.
``RelaxedLoss``  L(softmax(W / tau)) of the relaxation (Section 3.8) with its
                 exact gradient as the backward.

Both run entirely in libtenscol on the tensor's CUDA device; PyTorch only
holds the memory and orders the streams.
"""
from __future__ import annotations

import torch

from .tenscol import TensCol


class OneHotLoss(torch.autograd.Function):
    """forward(W, tc) -> L; the population of `tc` becomes W (same D, n, k)."""

    @staticmethod
    def forward(ctx, W: torch.Tensor, tc: TensCol):
        W = W.detach().contiguous()
        tc.tc_set_stream(torch.cuda.current_stream(W.device).cuda_stream)
        tc.tc_set_state_dev(W.data_ptr())
        grad = torch.empty_like(W)
        loss = torch.empty(3, dtype=torch.float32, device=W.device)
        tc.tc_st_grad_dev(grad.data_ptr(), loss.data_ptr())
        ctx.save_for_backward(grad)
        return loss[0].clone()

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None


class RelaxedLoss(torch.autograd.Function):
    """forward(W, tc, tau, t) -> L(softmax(W / tau)) with the graph and
    parameters of `tc`."""

    @staticmethod
    def forward(ctx, W: torch.Tensor, tc: TensCol, tau: float, t: int):
        W = W.detach().contiguous()
        tc.tc_set_stream(torch.cuda.current_stream(W.device).cuda_stream)
        grad = torch.empty_like(W)
        loss = torch.empty(4, dtype=torch.float32, device=W.device)
        tc.tc_relaxed_dev(W.data_ptr(), tau, t, loss.data_ptr(), grad.data_ptr())
        ctx.save_for_backward(grad)
        return loss[0].clone()

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        return g * grad, None, None, None
