"""The launch-shape table (bsi_set_tile_configs / bsi_get_tile_config) on the
CPU: validation, lookup, workspace sizes, and -- for many shapes -- the
host-side range check of every kernel access."""
import itertools

import numpy as np
import pytest

import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import bsi as B


@pytest.fixture(autouse=True)
def clean_table():
    B.bsi_set_tile_configs([])
    yield
    B.bsi_set_tile_configs([])


def test_defaults_and_lookup():
    d = B.bsi_get_tile_config((5, 5, 5))
    assert d == {"dx": 5, "dy": 5, "dz": 5, "adj_zchunk": 0, "adj_warps": 4, "fwd_strip_tiles": 0, "fwd_warps": 8}
    B.bsi_set_tile_configs([{"dx": 5, "dy": 5, "dz": 5, "adj_zchunk": 6},
                            {"dx": 3, "adj_zchunk": 8, "fwd_strip_tiles": 16},
                            {"adj_warps": 2}])
    assert B.bsi_get_tile_config((5, 5, 5))["adj_zchunk"] == 6
    assert B.bsi_get_tile_config((7, 9, 3))["fwd_strip_tiles"] == 16      # dx wildcard entry
    assert B.bsi_get_tile_config((7, 9, 4))["adj_warps"] == 2            # catch-all entry
    assert B.bsi_tile_configs()[1]["dx"] == 3


@pytest.mark.parametrize("bad", [{"adj_zchunk": 2}, {"adj_zchunk": 17}, {"fwd_strip_tiles": 3},
                                 {"fwd_strip_tiles": 30}, {"adj_warps": 5}, {"fwd_warps": -1}, {"dx": 65}])
def test_invalid_entries_rejected_and_table_kept(bad):
    B.bsi_set_tile_configs([{"adj_zchunk": 5}])
    with pytest.raises(B.BsiError):
        B.bsi_set_tile_configs([bad])
    assert B.bsi_get_tile_config((4, 4, 4))["adj_zchunk"] == 5


def test_too_many_entries_rejected():
    with pytest.raises(B.BsiError):
        B.bsi_set_tile_configs([{"adj_zchunk": 4}] * 257)


def test_workspace_follows_zchunk():
    shape, sp = (300, 512, 512), (5, 5, 5)
    sizes = []
    for zc in (3, 4, 8, 16):
        B.bsi_set_tile_configs([{"adj_zchunk": zc}])
        sizes.append(B.bsi_adjoint_workspace_bytes(shape, sp))
    assert sizes == sorted(sizes, reverse=True)   # longer chunks overlap less


SHAPES = [((37, 45, 61), (5, 4, 3)), ((20, 33, 170), (2, 3, 8)), ((9, 8, 140), (3, 5, 13)),
          ((16, 16, 96), (4, 4, 4)), ((11, 7, 300), (6, 5, 7))]


@pytest.mark.parametrize("zc,strip,w", list(itertools.product((3, 5, 16), (4, 17, 29), (0, 1, 3))))
def test_selfcheck_under_shapes(zc, strip, w):
    B.bsi_set_tile_configs([{"adj_zchunk": zc, "fwd_strip_tiles": strip, "adj_warps": w, "fwd_warps": w}])
    for op in ("forward", "forward_bf16", "adjoint"):
        n, msg = P.bsi_selfcheck_ranges([s for s, _ in SHAPES], [d for _, d in SHAPES], op, cover=True)
        assert n == 0, (op, msg)
