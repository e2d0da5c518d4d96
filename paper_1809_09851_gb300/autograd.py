"""Differentiable inviscid flux: forward = fdbb_flux, backward = fdbb_flux_vjp
(under a general EOS: fdbb_flux_eos and fdbb_flux_vjp_eos).

``flux(U, dir)`` returns the flux column F_dir(U) (nv tensors) and records a
``torch.autograd.Function`` whose backward evaluates the vector-Jacobian
product gU = A_dir(U)^T G in one kernel (no Jacobian is materialised).
``flux(U, dir, eos=...)`` does the same under a general equation of state
(a dict as in ``blocks.flux_eos``).

U may be a list of nv 1-D CUDA tensors or one (nv, N) tensor with contiguous
rows; the result has the same form.
"""
from __future__ import annotations

import torch

from . import blocks


class _Flux(torch.autograd.Function):
    @staticmethod
    def forward(ctx, dir: int, gamma: float, dw: bool, eos, *U):
        U = [u.contiguous() for u in U]
        if eos is None:
            F = blocks.flux(U, dir, gamma, dw=dw)
        else:
            F = blocks.flux_eos(U, eos, dir, dw=dw)
        ctx.save_for_backward(*U)
        ctx.dir, ctx.gamma, ctx.dw, ctx.eos = dir, gamma, dw, eos
        return tuple(F)

    @staticmethod
    def backward(ctx, *gF):
        U = list(ctx.saved_tensors)
        G = [torch.zeros_like(U[0]) if g is None else g.contiguous() for g in gF]
        if ctx.eos is None:
            gU = blocks.flux_vjp(U, G, ctx.dir, ctx.gamma, dw=ctx.dw)
        else:
            gU = blocks.flux_vjp_eos(U, G, ctx.eos, ctx.dir, dw=ctx.dw)
        return (None, None, None, None, *gU)


def flux(U, dir: int, gamma: float = blocks.GAMMA, dw: bool = False, eos=None):
    """Differentiable F_dir(U) (ideal gas with gamma, or the general EOS `eos`)."""
    if dir < 0:
        raise ValueError("the differentiable flux takes one direction (dir >= 0)")
    stacked = isinstance(U, torch.Tensor) and U.dim() == 2
    planes = list(U.unbind(0)) if stacked else list(U)
    out = _Flux.apply(dir, gamma, dw, eos, *planes)
    return torch.stack(out, 0) if stacked else list(out)
