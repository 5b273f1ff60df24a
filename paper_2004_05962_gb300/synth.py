"""Seeded synthetic inputs for the B-spline interpolation workloads.

This module holds no interpolation arithmetic: it only draws control grids,
voxel gradients, images and batch geometries from numpy's ``default_rng``.
Both the CUDA path and the FP64 oracle consume the same arrays it returns.

The paper measures on CT and MR registration pairs (Table 1, Sec. 4) that are
not available here; these generators stand in for them with volumes of the
same shape, spacings in the paper's 3..8 voxel range, and smooth displacement
grids of a few voxels' magnitude.

All control grids are drawn in FP64 and rounded once to FP32; that FP32 array
is what both sides see.
"""
from __future__ import annotations

import numpy as np


def grid_shape(shape, spacing):
    """Stored control-grid dims (nz, ny, nx) for volume (Z, Y, X) at spacing
    (dz, dy, dx): ceil(N/d) + 3 points per axis (a one-point border below,
    two above, so every 4x4x4 neighbourhood is in range)."""
    Z, Y, X = (int(s) for s in shape)
    dz, dy, dx = (int(s) for s in spacing)
    return (-(-Z // dz) + 3, -(-Y // dy) + 3, -(-X // dx) + 3)


def uniform_phi(shape, spacing, lo, hi, seed):
    """Control displacements i.i.d. uniform[lo, hi] voxels, FP32 [nz, ny, nx, 3]."""
    rng = np.random.default_rng(seed)
    g = grid_shape(shape, spacing)
    return rng.uniform(lo, hi, size=g + (3,)).astype(np.float32)


def gaussian_random_phi(shape, spacing, sigma_vox=3.0, smooth_cells=2.0, seed=2):
    """Smooth random control displacements (the CT-shaped workload).

    i.i.d. N(0, sigma_vox^2) per channel, a separable Gaussian filter of
    ``smooth_cells`` control cells (truncated at 4 sigma, reflecting border),
    then each channel rescaled so its standard deviation is ``sigma_vox``.
    """
    from scipy.ndimage import gaussian_filter1d

    rng = np.random.default_rng(seed)
    g = grid_shape(shape, spacing)
    a = rng.normal(0.0, sigma_vox, size=g + (3,))
    for axis in range(3):
        a = gaussian_filter1d(a, smooth_cells, axis=axis, mode="reflect", truncate=4.0)
    a *= sigma_vox / a.std(axis=(0, 1, 2), keepdims=True)
    return a.astype(np.float32)


def normal_field(shape, seed, scale=1.0):
    """Per-voxel, per-channel N(0, scale^2) FP32 array [Z, Y, X, 3] (the W of
    sum(W*u), or an incoming gradient for the adjoint)."""
    rng = np.random.default_rng(seed)
    Z, Y, X = (int(s) for s in shape)
    out = np.empty((Z, Y, X, 3), np.float32)
    # drawn slab by slab so that large volumes never hold an FP64 copy
    for z in range(Z):
        out[z] = rng.standard_normal((Y, X, 3), dtype=np.float32) * np.float32(scale)
    return out


def blob_params(shape, seed, nblobs=8, sigma_range=(8.0, 20.0)):
    """Centres (z, y, x), widths (voxels) and amplitudes of ``nblobs`` Gaussian
    blobs in a (Z, Y, X) volume: centres ~ U[0, N) per axis, widths ~ U[sigma_range],
    amplitudes ~ U[0.5, 1]."""
    rng = np.random.default_rng(seed)
    Z, Y, X = (int(s) for s in shape)
    out = []
    for _ in range(nblobs):
        c = rng.uniform([0, 0, 0], [Z, Y, X])
        s = rng.uniform(*sigma_range)
        a = rng.uniform(0.5, 1.0)
        out.append((c, s, a))
    return out


def blob_image(shape, seed, nblobs=8, sigma_range=(8.0, 20.0)):
    """A smooth FP32 image [Z, Y, X]: the sum of the blob_params blobs, each the
    product of three 1-D Gaussians (the isotropic Gaussian, separated)."""
    Z, Y, X = (int(s) for s in shape)
    img = np.zeros((Z, Y, X), np.float64)
    for c, s, a in blob_params(shape, seed, nblobs, sigma_range):
        ez = np.exp(-((np.arange(Z) - c[0]) ** 2) / (2 * s * s))
        ey = np.exp(-((np.arange(Y) - c[1]) ** 2) / (2 * s * s))
        ex = np.exp(-((np.arange(X) - c[2]) ** 2) / (2 * s * s))
        img += a * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return img.astype(np.float32)


def batch_geometries(n=64, seed=5, xy_range=(48, 256), z_range=(48, 160), spacing_range=(3, 8)):
    """Uneven registration batch: ``n`` volumes with X, Y ~ U_int[48, 256],
    Z ~ U_int[48, 160] and each spacing axis ~ U_int[3, 8].

    Returns a list of ((Z, Y, X), (dz, dy, dx)) tuples.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        X = int(rng.integers(xy_range[0], xy_range[1] + 1))
        Y = int(rng.integers(xy_range[0], xy_range[1] + 1))
        Z = int(rng.integers(z_range[0], z_range[1] + 1))
        d = rng.integers(spacing_range[0], spacing_range[1] + 1, size=3)
        out.append(((Z, Y, X), (int(d[2]), int(d[1]), int(d[0]))))
    return out


def sample_voxels(shape, n, seed):
    """``n`` distinct-ish voxel indices [n, 3] as (x, y, z), including the eight
    corners of the volume so that both borders are always covered."""
    rng = np.random.default_rng(seed)
    Z, Y, X = (int(s) for s in shape)
    pts = np.stack([rng.integers(0, X, n), rng.integers(0, Y, n), rng.integers(0, Z, n)], axis=1)
    corners = np.array([[x, y, z] for x in (0, X - 1) for y in (0, Y - 1) for z in (0, Z - 1)])
    return np.concatenate([corners, pts]).astype(np.int64)


def sample_grid_points(grid, n, seed):
    """``n`` stored control points [n, 3] as (gx, gy, gz) of a grid (nz, ny, nx),
    including its eight corners."""
    rng = np.random.default_rng(seed)
    nz, ny, nx = grid
    pts = np.stack([rng.integers(0, nx, n), rng.integers(0, ny, n), rng.integers(0, nz, n)], axis=1)
    corners = np.array([[x, y, z] for x in (0, nx - 1) for y in (0, ny - 1) for z in (0, nz - 1)])
    return np.concatenate([corners, pts]).astype(np.int64)
