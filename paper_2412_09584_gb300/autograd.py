"""alpha-CROWN under torch.autograd: the CROWN lower bound as a differentiable function of the slopes and of the
box.

The free lower slopes alpha of Lemma 1 (Appendix B.1) make the bound a function LB(alpha); its gradient is
computed by the hand-written adjoint in libbab (`bab_alpha_grad`: a forward pass of the relaxed network at the
concretizing point).  `CrownBound.apply(alpha, problem)` returns the per-box bounds and lets any torch
optimiser raise them; the library call computes the bound and the gradient together, and backward scales the
stored gradient by the incoming one.  `CrownBoxBound.apply(lo, hi, problem, alpha)` does the same for the box
faces (`bab_box_grad`: the relaxed network's sensitivities carried back through the interval bounds).  Only
argument marshalling happens here.
"""
from __future__ import annotations

import torch

from . import binding as B


class CrownProblem:
    """A context plus the problem and boxes the bound is taken over (all CUDA tensors)."""

    def __init__(self, ctx, x0, goal, horizon, rho, lo, hi, precision=B.PREC_FP32):
        self.ctx, self.x0, self.goal = ctx, x0, goal
        self.horizon, self.rho, self.lo, self.hi = int(horizon), float(rho), lo, hi
        self.precision = precision


class CrownBound(torch.autograd.Function):
    """lb = CROWN bound of each box at slopes alpha [n, H, sumh]; d lb / d alpha from the library adjoint."""

    @staticmethod
    def forward(ctx, alpha, prob: CrownProblem):
        a = alpha.detach().contiguous()
        n = a.shape[0]
        lb = torch.empty(n, device=a.device, dtype=torch.float32)
        grad = torch.empty_like(a)
        B.bab_alpha_grad(prob.ctx, prob.x0, prob.goal, prob.horizon, prob.rho, prob.lo, prob.hi, n, a, lb, grad,
                         precision=prob.precision)
        ctx.save_for_backward(grad)
        return lb

    @staticmethod
    def backward(ctx, grad_lb):
        (grad,) = ctx.saved_tensors
        return grad * grad_lb.reshape(-1, *([1] * (grad.dim() - 1))), None


def crown_bound(alpha, prob: CrownProblem):
    return CrownBound.apply(alpha, prob)


class CrownBoxBound(torch.autograd.Function):
    """lb = FP32 CROWN bound of each box [lo, hi] at fixed slopes alpha (None: adaptive); d lb / d lo and
    d lb / d hi from the library adjoint.  prob.lo / prob.hi are not used: the faces are the arguments."""

    @staticmethod
    def forward(ctx, lo, hi, prob: CrownProblem, alpha=None):
        lo_, hi_ = lo.detach().contiguous(), hi.detach().contiguous()
        n = lo_.shape[0]
        lb = torch.empty(n, device=lo_.device, dtype=torch.float32)
        glo, ghi = torch.empty_like(lo_), torch.empty_like(hi_)
        a = None if alpha is None else alpha.detach().contiguous()
        B.bab_box_grad(prob.ctx, prob.x0, prob.goal, prob.horizon, prob.rho, lo_, hi_, n, lb, glo, ghi, alpha=a)
        ctx.save_for_backward(glo, ghi)
        return lb

    @staticmethod
    def backward(ctx, grad_lb):
        glo, ghi = ctx.saved_tensors
        w = grad_lb.reshape(-1, 1)
        return glo * w, ghi * w, None, None


def crown_box_bound(lo, hi, prob: CrownProblem, alpha=None):
    return CrownBoxBound.apply(lo, hi, prob, alpha)
