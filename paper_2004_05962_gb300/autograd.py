"""Differentiable B-spline interpolation: ``field(phi, shape, spacing)``.

Forward is ``bsi_field_forward`` (Eq. 1, Sec. 2.1); backward is the
hand-written adjoint ``bsi_field_adjoint`` (the transpose of Eq. 1, which
gathers dL/dfield back onto the control points -- the step every gradient
iteration of the FFD registration loop performs).
"""
from __future__ import annotations

import torch

from .bsi import (bsi_field_adjoint, bsi_field_adjoint_rational, bsi_field_forward, bsi_field_forward_rational,
                  bsi_resample_backward, bsi_resample_forward)


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


class BSIFieldRational(torch.autograd.Function):
    """Eq. 1 on a grid of non-integer spacing num/den with lattice shift off/den
    per axis: forward ``bsi_field_forward_rational``, backward its transpose
    ``bsi_field_adjoint_rational``."""

    @staticmethod
    def forward(ctx, phi, shape, num, den, off):
        ctx.rat = (tuple(int(v) for v in num), tuple(int(v) for v in den), tuple(int(v) for v in off))
        return bsi_field_forward_rational(phi.contiguous(), shape, *ctx.rat)

    @staticmethod
    def backward(ctx, grad_field):
        g = grad_field.contiguous()
        if g.dtype != torch.float32:
            g = g.float()
        return bsi_field_adjoint_rational(g, *ctx.rat), None, None, None, None


def field_rational(phi: torch.Tensor, shape, num, den, off=(0, 0, 0)) -> torch.Tensor:
    """Dense displacement field [Z, Y, X, 3] from a control grid of spacing
    num/den voxels and lattice shift off/den voxels per axis ((z, y, x) order
    like ``shape``), differentiable in phi."""
    return BSIFieldRational.apply(phi, tuple(int(s) for s in shape), num, den, off)


class BSIResample(torch.autograd.Function):
    """Floating image resampled by the BSI displacement, without storing the
    field: forward ``bsi_resample_forward``, backward (with respect to phi only)
    ``bsi_resample_backward``."""

    @staticmethod
    def forward(ctx, phi, image, shape, spacing):
        ctx.shape = tuple(int(s) for s in shape)
        ctx.spacing = tuple(int(s) for s in spacing)
        phi, image = phi.contiguous(), image.contiguous()
        ctx.save_for_backward(phi, image)
        return bsi_resample_forward(phi, ctx.shape, ctx.spacing, image)

    @staticmethod
    def backward(ctx, grad_warped):
        phi, image = ctx.saved_tensors
        g = grad_warped.contiguous()
        if g.dtype != torch.float32:
            g = g.float()
        return bsi_resample_backward(phi, ctx.shape, ctx.spacing, image, g), None, None, None


def resample(phi: torch.Tensor, image: torch.Tensor, shape, spacing) -> torch.Tensor:
    """Floating ``image`` [fZ, fY, fX] sampled at x + T(x) for every voxel x of a
    (Z, Y, X) = ``shape`` volume, T the BSI displacement of ``phi`` (trilinear,
    zeros outside the image); differentiable in phi."""
    return BSIResample.apply(phi, image, tuple(int(s) for s in shape), tuple(int(s) for s in spacing))
