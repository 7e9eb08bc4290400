"""torch.autograd wrapper of the fidelity-gradient kernel.

    F = PostSelectedFidelity.apply(theta, circ, n_patterns, first_pattern, seed, precision)

returns the post-selected output fidelity of each fixed error pattern (a
float64 CUDA tensor); F.backward(w) accumulates sum_p w_p dF_p/dtheta into
theta.grad. Patterns with zero acceptance contribute F = 0 and no gradient.
"""
from __future__ import annotations

import torch

from . import soft_fidelity_grad


class PostSelectedFidelity(torch.autograd.Function):
    @staticmethod
    def forward(ctx, theta, circ, n_patterns, first_pattern=0, seed=0, precision="fp64"):
        th = theta.detach().to("cpu", torch.float64).numpy()
        fid, pacc, grad, status = soft_fidelity_grad(circ, th, n_patterns, first_pattern, seed, precision)
        ctx.save_for_backward(grad)
        ctx.theta_dtype = theta.dtype
        ctx.theta_device = theta.device
        ctx.mark_non_differentiable(pacc, status)
        return fid, pacc, status

    @staticmethod
    def backward(ctx, g_fid, g_pacc, g_status):
        (grad,) = ctx.saved_tensors
        gt = (g_fid.to(grad.dtype).unsqueeze(1) * grad).sum(0)
        return gt.to(ctx.theta_device, ctx.theta_dtype), None, None, None, None, None
