"""torch.autograd interface of the linewidth (Eq. linewidthel) and its adjoint.

``linewidth(model, g, T, EF, k, q, ...)`` returns Im Sigma_nk [nk, nw] as a
differentiable function of the Wannier-space vertex g(Re,Rp) (complex128 CUDA
tensor with the model's g layout), the temperature T and the Fermi level E_F
(0-dim float64 tensors).  The backward pass calls epw_linewidth_backward, which
recomputes g(k,q) instead of storing it; the gradient with respect to g follows
torch's convention for complex inputs (dL/dRe g + i dL/dIm g).

T and E_F enter the kernels as host scalars: their values are read once in the
forward (free for CPU tensors, one device read for CUDA tensors) and kept for
the backward, which reads nothing back from the device.  The model is the
vertex's owner on the device: after a call its vertex is g (the upload is
skipped when the model already holds this tensor at this version).
"""
from __future__ import annotations

import weakref

import torch

from .api import FP64


def _host_scalar(x) -> float:
    """Value of a 0-dim tensor (or number) on the host; one device read for a CUDA tensor."""
    if isinstance(x, torch.Tensor):
        return float(x.detach().cpu()) if x.is_cuda else float(x.detach())
    return float(x)


def _load_vertex(model, g):
    """Upload g unless the model already holds this tensor (same object, same version)."""
    held = getattr(model, "_autograd_vertex", None)
    if held is None or held[0]() is not g or held[1] != g._version:
        model.set_vertex(g.detach())
        model._autograd_vertex = (weakref.ref(g), g._version)


class LinewidthFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, g, T, EF, model, k, q, wq, sigma, omega_min, precision):
        Th, EFh = _host_scalar(T), _host_scalar(EF)
        _load_vertex(model, g)
        out = model.linewidth(k, q, wq, T=Th, EF=EFh, sigma=sigma, omega_min=omega_min, precision=precision)
        ctx.save_for_backward(g, T, EF)
        ctx.model = model
        ctx.args = (k, q, wq, sigma, omega_min, precision, Th, EFh)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        g, T, EF = ctx.saved_tensors
        k, q, wq, sigma, omega_min, precision, Th, EFh = ctx.args
        model = ctx.model
        _load_vertex(model, g)  # the model may have seen another vertex since forward
        dg, dT, dE = model.linewidth_backward(k, q, grad_out.detach().contiguous(), wq, T=Th, EF=EFh,
                                              sigma=sigma, omega_min=omega_min, precision=precision,
                                              want_dg=ctx.needs_input_grad[0])
        gT = torch.tensor(dT, dtype=T.dtype, device=T.device) if ctx.needs_input_grad[1] else None
        gE = torch.tensor(dE, dtype=EF.dtype, device=EF.device) if ctx.needs_input_grad[2] else None
        return dg, gT, gE, None, None, None, None, None, None, None


def linewidth(model, g, T, EF, k, q, wq=None, *, sigma: float, omega_min: float = 1e-5, precision: int = FP64):
    """Differentiable Im Sigma_nk [nk, nw]; see the module docstring."""
    return LinewidthFn.apply(g, T, EF, model, k, q, wq, sigma, omega_min, precision)
