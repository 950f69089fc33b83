"""torch.autograd interface of the linewidth (Eq. linewidthel) and its adjoint.

``linewidth(model, g, T, EF, k, q, ...)`` returns Im Sigma_nk [nk, nw] as a
differentiable function of the Wannier-space vertex g(Re,Rp) (complex128 CUDA
tensor with the model's g layout), the temperature T and the Fermi level E_F
(0-dim float64 tensors).  The backward pass calls epw_linewidth_backward, which
recomputes g(k,q) instead of storing it; the gradient with respect to g follows
torch's convention for complex inputs (dL/dRe g + i dL/dIm g).
"""
from __future__ import annotations

import torch

from .api import FP64


class LinewidthFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, T, EF, model, k, q, wq, sigma, omega_min, precision):
        model.set_vertex(g.detach())
        out = model.linewidth(k, q, wq, T=float(T), EF=float(EF), sigma=sigma, omega_min=omega_min,
                              precision=precision)
        ctx.save_for_backward(g, T, EF)
        ctx.model = model
        ctx.args = (k, q, wq, sigma, omega_min, precision)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g, T, EF = ctx.saved_tensors
        k, q, wq, sigma, omega_min, precision = ctx.args
        model = ctx.model
        model.set_vertex(g.detach())  # the model may have seen another vertex since forward
        dg, dT, dE = model.linewidth_backward(k, q, grad_out.detach().contiguous(), wq, T=float(T), EF=float(EF),
                                              sigma=sigma, omega_min=omega_min, precision=precision,
                                              want_dg=ctx.needs_input_grad[0])
        gT = torch.tensor(dT, dtype=T.dtype, device=T.device) if ctx.needs_input_grad[1] else None
        gE = torch.tensor(dE, dtype=EF.dtype, device=EF.device) if ctx.needs_input_grad[2] else None
        return dg, gT, gE, None, None, None, None, None, None, None


def linewidth(model, g, T, EF, k, q, wq=None, *, sigma: float, omega_min: float = 1e-5, precision: int = FP64):
    """Differentiable Im Sigma_nk [nk, nw]; see the module docstring."""
    return LinewidthFn.apply(g, T, EF, model, k, q, wq, sigma, omega_min, precision)
