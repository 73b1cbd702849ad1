"""The dual function g(lambda, p, B) of Eq. (5) as a torch.autograd.Function.

Forward runs the user pass (Algorithm 1 for every user, Algorithm 2's
reduce) in the CUDA library; backward runs the library's gradient kernel,
which applies Danskin's theorem at the maximiser x*:
    dg/dlambda_k = B_k - R_k,   dg/dp_ij = x*_ij,   dg/dB_k = lambda_k,
each scaled by the upstream gradient inside the kernel.  The paper states no
gradient; this is the derivative of its dual, valid wherever x* is unique
(away from the breakpoints where two items tie).
"""
from __future__ import annotations

import torch

from . import kp


class DualFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, lam: torch.Tensor, p: torch.Tensor, B: torch.Tensor, prob: "kp.Problem"):
        if p.data_ptr() != prob._keep[0].data_ptr() or B.data_ptr() != prob._keep[1].data_ptr():
            raise ValueError("p and B must be the tensors the problem was created with")
        lam = lam.detach().contiguous()
        R = torch.empty(prob.K, dtype=torch.float64, device=lam.device)
        g = torch.empty((), dtype=torch.float64, device=lam.device)
        x = torch.empty(prob.N * prob.W, dtype=torch.int32, device=lam.device)
        kp.kp_reduce_consumption(prob, lam, R=R, g=g, x_bits=x)
        ctx.save_for_backward(lam, x, R)
        ctx.prob = prob
        ctx.p_shape = p.shape
        return g

    @staticmethod
    def backward(ctx, grad_g):
        lam, x, R = ctx.saved_tensors
        prob = ctx.prob
        up = grad_g.detach().to(torch.float64).reshape(()).contiguous()
        need_l, need_p, need_B = ctx.needs_input_grad[:3]
        gl = torch.empty(prob.K, dtype=torch.float64, device=lam.device) if need_l else None
        gp = torch.empty(prob.N * prob.M, dtype=torch.float32, device=lam.device) if need_p else None
        gB = torch.empty(prob.K, dtype=torch.float64, device=lam.device) if need_B else None
        if need_l or need_p or need_B:
            kp.kp_dual_backward(prob, lam, x, R, up, grad_lambda=gl, grad_p=gp, grad_B=gB)
        return gl, (gp.view(ctx.p_shape) if gp is not None else None), gB, None


def dual(lam: torch.Tensor, prob: "kp.Problem") -> torch.Tensor:
    """g(lambda) with gradients to lambda, p and B (the problem's own tensors)."""
    p, B = prob._keep[0], prob._keep[1]
    return DualFunction.apply(lam, p, B, prob)
