"""The App. A / App. B analytic models against the figures the paper prints."""
import os

import pytest

from paper_2004_05962_gb300 import model

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _figures():
    out = {}
    with open(os.path.join(GOLDEN, "paper_appendix_figures.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            key, val, tol = line.split()[:3]
            out[key] = (float(val), float(tol))
    return out


FIG = _figures()


def test_transfer_ratios_at_5cubed():
    M, T = 125 * 1000, 125          # any volume; 5x5x5 tiles
    tt = model.transfers_blocks_of_tiles(M, T, 4, 4, 4)   # 4x4x4 tiles per block
    v, tol = FIG["transfer_ratio_vs_block_per_tile_at_5cubed"]
    assert abs(model.transfers_block_per_tile(M, T) / tt - v) <= tol
    v, tol = FIG["transfer_ratio_vs_texture_at_5cubed"]
    assert abs(model.transfers_texture(M) / tt - v) <= tol
    # observation 1 of App. A: texture beats no-tiles; observation 2: block per tile beats texture for T > 8
    assert model.transfers_texture(M) < model.transfers_no_tiles(M)
    assert model.transfers_block_per_tile(M, 9) < model.transfers_texture(M)


def test_operation_counts():
    assert model.ops_direct_triple_sum() == FIG["ops_per_voxel_direct_triple_sum"][0]
    assert model.ops_fused_weight() == FIG["ops_per_voxel_fused_weight"][0]
    assert model.ops_trilinear() == FIG["ops_per_voxel_trilinear"][0]


def test_separable_fma_counts():
    # per voxel, 3 channels, one cell: 3 * (4 + 16/dx + 64/(dx*dy))
    assert model.fma_separable_per_voxel(5, 5, 5) == pytest.approx(29.28)
    assert model.fma_separable_per_voxel(3, 3, 3) == pytest.approx(3 * (4 + 16 / 3 + 64 / 9))
    # a warp computes 32 columns for 29 cells of one y-cell: z and y stages shrink
    want = 12 * 32 * 4 / (29 * 25) + 12 * 32 / (29 * 5) + 12
    assert model.fma_separable_per_voxel(5, 5, 5, cells_x=29) == pytest.approx(want)


def test_algorithmic_bytes():
    shape, spacing = (300, 512, 512), (5, 5, 5)
    b = model.forward_bytes(shape, spacing)
    assert b == 300 * 512 * 512 * 12 + 63 * 106 * 106 * 12
    assert model.forward_bytes(shape, spacing, 2) == 300 * 512 * 512 * 6 + 63 * 106 * 106 * 12
    assert model.adjoint_bytes(shape, spacing) == b
    assert model.grid_points((64, 64, 64), (5, 5, 5)) == 16 ** 3
