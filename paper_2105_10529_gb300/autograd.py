"""torch.autograd front ends of the derivative kernels.

cross_section(mt, alpha_s, ...) is the Monte Carlo estimate of sigma at a
fixed VEGAS grid and fixed random numbers: its forward call runs one VEGAS
pass; its backward call runs the derivative pass, which recomputes every
event (kinematics, PDFs, matrix element) with forward-mode derivatives and
stores nothing between the two calls.  The cut masks are those of the base
point, so the gradient is the pathwise derivative of the estimate.

matrix_element(momenta, ...) is |M|^2 of given momenta; its backward call
returns d|M|^2/dp from the derivative kernel.
"""
from __future__ import annotations

import torch

from .api import Context


class _CrossSection(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mt, alpha_s, context: Context, process: int, sqrt_s: float, grid, n_events: int, iteration: int):
        context.set_couplings(float(mt), float(alpha_s))
        sums, _ = context.vegas_pass(process, sqrt_s, grid, n_events, iteration=iteration)
        ctx.args = (context, process, sqrt_s, grid, n_events, iteration, float(mt), float(alpha_s))
        return sums[0].clone()

    @staticmethod
    def backward(ctx, g):
        context, process, sqrt_s, grid, n_events, iteration, mt, alpha_s = ctx.args
        context.set_couplings(mt, alpha_s)
        d = context.vegas_pass_grad(process, sqrt_s, grid, n_events, iteration=iteration)
        return g * d[1], g * d[3], None, None, None, None, None, None


def cross_section(mt, alpha_s, context: Context, process: int, sqrt_s: float, grid, n_events: int,
                  iteration: int = 0):
    """sigma_hat(m_t, alpha_s) in pb, differentiable in m_t and alpha_s."""
    return _CrossSection.apply(mt, alpha_s, context, process, sqrt_s, grid, n_events, iteration)


class _MatrixElement(torch.autograd.Function):
    @staticmethod
    def forward(ctx, momenta, context: Context, process: int):
        ctx.args = (context, process)
        ctx.save_for_backward(momenta)
        return context.evaluate(process, momenta)

    @staticmethod
    def backward(ctx, g):
        context, process = ctx.args
        (momenta,) = ctx.saved_tensors
        _, dme = context.evaluate_grad(process, momenta)
        return g[:, None, None] * dme, None, None


def matrix_element(momenta, context: Context, process: int):
    """Averaged |M|^2 of momenta [n, n_ext, 4], differentiable in the momenta."""
    return _MatrixElement.apply(momenta, context, process)
