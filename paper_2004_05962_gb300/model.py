"""Traffic and operation-count models of B-spline interpolation.

Two uses:
  * the paper's analytic models, restated from App. A (off-chip transfer counts,
    Eqs. A1-A4) and App. B (operations per voxel), pinned in the tests against
    the figures the paper prints (about 12x and 187x fewer transfers at 5^3
    tiles, Sec. 3.2.1; 255, 127 and 126 operations per voxel, App. B);
  * the ALGORITHMIC bytes per voxel that the benchmark divides by the measured
    kernel time to report achieved HBM bandwidth.  Algorithmic bytes count each
    input read once and each output written once; workspace partials and
    re-reads are implementation traffic and are not counted.
"""
from __future__ import annotations

import math

# --- App. A: off-chip -> on-chip transfers (in L-word transactions) ----------


def transfers_no_tiles(M, N=64, L=1):
    """Eq. A1: every voxel fetches its N control points."""
    return N * M / L


def transfers_texture(M, L=1):
    """Eq. A2: hardware trilinear filtering fetches 2^3 values per voxel."""
    return 8 * M / L


def transfers_block_per_tile(M, T, N=64, L=1):
    """Eq. A3: each tile of T voxels fetches its N control points once."""
    return N * M / (T * L)


def transfers_blocks_of_tiles(M, T, l, m, n, L=1):
    """Eq. A4: a block of l x m x n tiles fetches its (3+l)(3+m)(3+n) points once."""
    return (3 + l) * (3 + m) * (3 + n) * M / (l * m * n * T * L)


# --- App. B: arithmetic operations per voxel (per vector channel) -------------


def ops_direct_triple_sum():
    """Eq. 1 with three separate weights per summand: 64 * (3 mul + 1 add) - 1."""
    return 64 * (3 + 1) - 1


def ops_fused_weight():
    """Eq. 1 with one precomputed weight per summand: 64 * (1 mul + 1 add) - 1."""
    return 64 * (1 + 1) - 1


def ops_trilinear():
    """The 8+1 trilinear rewrite: 9 cubes x 7 lerps x 2 operations."""
    return 9 * 7 * 2


def fma_separable_per_voxel(dx, dy, dz, channels=3, cells_x=None, cells_y=None):
    """FMAs per voxel of the separable (z, then y, then x) contraction used by
    the CUDA kernels: 4 taps per axis, z-stage amortised over the dy*dx voxels
    of a column and y-stage over the dx voxels of a row.  With ``cells_x`` /
    ``cells_y`` the z and y stages are shared by that many neighbouring cells
    (the x-group of a warp), otherwise one cell is assumed."""
    if cells_x is None:
        return channels * (4 + 16 / dx + 64 / (dx * dy))
    cy = cells_y or 1
    zstage = 12 * (cells_x + 3) * (cy + 3) / (cells_x * cy * dx * dy)
    ystage = 12 * (cells_x + 3) / (cells_x * dx)
    return zstage * channels / 3 + ystage * channels / 3 + 4 * channels


# --- algorithmic bytes ----------------------------------------------------------


def grid_points(shape, spacing):
    Z, Y, X = shape
    dz, dy, dx = spacing
    return (math.ceil(Z / dz) + 3) * (math.ceil(Y / dy) + 3) * (math.ceil(X / dx) + 3)


def forward_bytes(shape, spacing, out_bytes_per_channel=4):
    """Forward: write the 3-channel field once, read the FP32 grid once."""
    Z, Y, X = shape
    return Z * Y * X * 3 * out_bytes_per_channel + grid_points(shape, spacing) * 12


def adjoint_bytes(shape, spacing):
    """Adjoint: read the FP32 3-channel voxel gradient once, write the grid gradient once."""
    Z, Y, X = shape
    return Z * Y * X * 12 + grid_points(shape, spacing) * 12


def resample_bytes(shape, spacing, fshape=None, out_bytes=4):
    """Algorithmic bytes of the fused BSI + resampling forward: the floating
    image read once (4 B per element), the warped image written once, the
    control grid read once.  The displacement field is never stored."""
    fshape = shape if fshape is None else fshape
    return 4 * math.prod(fshape) + out_bytes * math.prod(shape) + 12 * grid_points(shape, spacing)


def resample_backward_bytes(shape, spacing, fshape=None):
    """Algorithmic bytes of its gradient with respect to phi: the floating image
    and dL/dwarped read once, the control grid read and dL/dphi written once
    (the voxel gradient G that the implementation passes from its first stage
    to the adjoint is extra)."""
    fshape = shape if fshape is None else fshape
    return 4 * math.prod(fshape) + 4 * math.prod(shape) + 24 * grid_points(shape, spacing)
