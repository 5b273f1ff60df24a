"""The autotuner and non-default launch shapes on the GPU: results match the
FP64 oracle under every shape, and a tuning run installs a valid table."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import bsi as B
from paper_2004_05962_gb300 import synth, tune
from gpu_util import ADJ_TOL, FWD_TOL, adj_err, dev, fwd_err, gpu_adjoint, gpu_forward

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def clean_table():
    B.bsi_set_tile_configs([])
    yield
    B.bsi_set_tile_configs([])


@pytest.mark.parametrize("cfg", [{"adj_zchunk": 3, "fwd_strip_tiles": 16, "adj_warps": 4, "fwd_warps": 4},
                                 {"adj_zchunk": 8, "fwd_strip_tiles": 5, "adj_warps": 1, "fwd_warps": 2},
                                 {"adj_zchunk": 16, "fwd_strip_tiles": 29}])
def test_parity_under_nondefault_shapes(cfg):
    B.bsi_set_tile_configs([cfg])
    for shape, spacing in [((37, 45, 61), (5, 4, 3)), ((20, 33, 170), (2, 3, 8)), ((9, 8, 140), (3, 5, 13))]:
        phi = synth.uniform_phi(shape, spacing, -2, 2, seed=90)
        err, tol = fwd_err(gpu_forward(phi, shape, spacing), phi, shape, spacing)
        assert err <= tol, (cfg, shape, spacing)
        g = synth.normal_field(shape, seed=91)
        err, tol = adj_err(gpu_adjoint(g, spacing), g, spacing)
        assert err <= tol, (cfg, shape, spacing)


def test_tuning_run_installs_valid_table(tmp_path):
    shapes = [(40, 64, 96), (48, 80, 64)]
    spacings = [(5, 5, 5), (4, 3, 6)]
    entries = tune.tune(spacings, shapes, cache_path=tmp_path / "cache.json", iters=2)
    assert len(entries) == 2
    assert (tmp_path / "cache.json").exists()
    for e, sp in zip(entries, spacings):
        assert (e["dz"], e["dy"], e["dx"]) == sp
        assert 3 <= e["adj_zchunk"] <= 16
    # a second call loads from the cache without re-timing and gives the same table
    assert tune.tune(spacings, shapes, cache_path=tmp_path / "cache.json") == entries
    for shape, spacing in zip(shapes, spacings):
        phi = synth.uniform_phi(shape, spacing, -2, 2, seed=92)
        err, tol = fwd_err(gpu_forward(phi, shape, spacing), phi, shape, spacing)
        assert err <= tol


def test_tune_batched_single_shape_for_the_launch(tmp_path):
    geoms = synth.batch_geometries(6, seed=93, xy_range=(16, 64), z_range=(16, 32))
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    e = tune.tune_batched(shapes, spacings, cache_path=tmp_path / "c.json", iters=2)
    assert (e["dx"], e["dy"], e["dz"]) == (0, 0, 0)          # one wildcard entry for the whole launch
    assert 3 <= e["adj_zchunk"] <= 16 and B.bsi_tile_configs() == [e]
    phis = [synth.uniform_phi(s, d, -2, 2, seed=94 + i) for i, (s, d) in enumerate(geoms)]
    outs = P.bsi_field_forward_batched([torch.from_numpy(p).to(dev()) for p in phis], shapes, spacings)
    grads = [synth.normal_field(s, seed=95 + i) for i, s in enumerate(shapes)]
    dps = P.bsi_field_adjoint_batched([torch.from_numpy(g).to(dev()) for g in grads], spacings)
    torch.cuda.synchronize()
    for i, (s, d) in enumerate(geoms):
        err, tol = fwd_err(outs[i], phis[i], s, d)
        assert err <= tol
        err, tol = adj_err(dps[i], grads[i], d)
        assert err <= tol
