"""PyTorch autograd wrappers of the holographic forward model and its adjoint.

``HologramModel.apply(x, h)`` returns ``H x`` (librihv's rihv_forward) and its
backward applies the hand-written adjoint kernel (rihv_adjoint);
``HologramAdjoint.apply(r, h)`` is the transpose pair. Both are C-linear, so
with PyTorch's convention (the incoming gradient is dL/d(conj y)) the backward
of ``y = H x`` is ``H^H g`` and that of ``z = H^H r`` is ``H g``.

Work is queued on the stream that is current when the op runs, so the library
calls are ordered with the surrounding PyTorch work.
"""
from __future__ import annotations

import torch

from .rihv import Rihv


def _on_current_stream(h: Rihv):
    h.set_stream(torch.cuda.current_stream())


class HologramModel(torch.autograd.Function):
    """y = H x for x complex64 [nz][ny][nx] on the GPU; y complex64 [ny][nx]."""

    @staticmethod
    def forward(ctx, x: torch.Tensor, h: Rihv):
        if x.dtype != torch.complex64 or not x.is_cuda:
            raise TypeError("x must be a complex64 CUDA tensor")
        x = x.contiguous()
        out = torch.empty((h.ny, h.nx), dtype=torch.complex64, device=x.device)
        _on_current_stream(h)
        h.forward(x, out)
        ctx.h = h
        return out

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        h = ctx.h
        g = g.contiguous().to(torch.complex64)
        gx = torch.empty((h.nz, h.ny, h.nx), dtype=torch.complex64, device=g.device)
        _on_current_stream(h)
        h.adjoint(g, gx)
        return gx, None


class HologramAdjoint(torch.autograd.Function):
    """z = H^H r for r complex64 [ny][nx]; z complex64 [nz][ny][nx]."""

    @staticmethod
    def forward(ctx, r: torch.Tensor, h: Rihv):
        if r.dtype != torch.complex64 or not r.is_cuda:
            raise TypeError("r must be a complex64 CUDA tensor")
        r = r.contiguous()
        out = torch.empty((h.nz, h.ny, h.nx), dtype=torch.complex64, device=r.device)
        _on_current_stream(h)
        h.adjoint(r, out)
        ctx.h = h
        return out

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        h = ctx.h
        g = g.contiguous().to(torch.complex64)
        gr = torch.empty((h.ny, h.nx), dtype=torch.complex64, device=g.device)
        _on_current_stream(h)
        h.forward(g, gr)
        return gr, None


def hologram_model(x: torch.Tensor, h: Rihv) -> torch.Tensor:
    return HologramModel.apply(x, h)


def hologram_adjoint(r: torch.Tensor, h: Rihv) -> torch.Tensor:
    return HologramAdjoint.apply(r, h)
