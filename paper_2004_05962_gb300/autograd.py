"""Differentiable B-spline interpolation: ``field(phi, shape, spacing)``.

Forward is ``bsi_field_forward`` (Eq. 1, Sec. 2.1); backward is the
hand-written adjoint ``bsi_field_adjoint`` (the transpose of Eq. 1, which
gathers dL/dfield back onto the control points -- the step every gradient
iteration of the FFD registration loop performs).
"""
from __future__ import annotations

import torch

from .bsi import bsi_field_adjoint, bsi_field_forward


class BSIField(torch.autograd.Function):
    @staticmethod
    def forward(ctx, phi, shape, spacing):
        ctx.spacing = tuple(int(s) for s in spacing)
        return bsi_field_forward(phi.contiguous(), shape, ctx.spacing)

    @staticmethod
    def backward(ctx, grad_field):
        g = grad_field.contiguous()
        if g.dtype != torch.float32:
            g = g.float()
        return bsi_field_adjoint(g, ctx.spacing), None, None


def field(phi: torch.Tensor, shape, spacing) -> torch.Tensor:
    """Dense displacement field [Z, Y, X, 3] from control grid phi [nz, ny, nx, 3]
    (shape = (Z, Y, X), spacing = (dz, dy, dx) voxels), differentiable in phi."""
    return BSIField.apply(phi, tuple(int(s) for s in shape), tuple(int(s) for s in spacing))
