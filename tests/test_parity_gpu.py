"""CUDA path vs FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import (ADJ_TOL, BF16_REL, FWD_TOL, adj_err, dev, fwd_err, gpu_adjoint,
                      gpu_forward)

pytestmark = pytest.mark.gpu

# (shape (Z, Y, X), spacing (dz, dy, dx)): several tiles, ragged tails, every
# specialised x-spacing 1..8, generic x-spacings, thin volumes, several x-groups
SMALL = [
    ((64, 64, 64), (5, 5, 5)),
    ((1, 1, 1), (1, 1, 1)),
    ((2, 3, 5), (1, 1, 1)),
    ((9, 10, 11), (2, 2, 2)),
    ((13, 7, 40), (3, 2, 3)),
    ((17, 19, 23), (4, 4, 4)),
    ((20, 11, 93), (6, 5, 5)),
    ((12, 13, 100), (5, 6, 6)),
    ((15, 9, 97), (7, 3, 7)),
    ((16, 16, 250), (8, 8, 8)),
    ((11, 12, 300), (4, 3, 9)),
    ((9, 8, 140), (3, 5, 13)),
    ((5, 4, 130), (2, 2, 64)),
    ((1, 40, 37), (3, 7, 4)),
    ((33, 1, 1), (5, 1, 1)),
    ((6, 7, 29 * 3 * 2 + 5), (2, 3, 2)),
]


@pytest.mark.parametrize("shape,spacing", SMALL, ids=[f"{s}-{d}" for s, d in SMALL])
def test_forward_f32_matches_oracle(shape, spacing):
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=sum(shape) + sum(spacing))
    got = gpu_forward(phi, shape, spacing)
    err, tol = fwd_err(got, phi, shape, spacing)
    assert err <= tol, (err, tol)


def test_forward_config_64cubed_seed1():
    """64^3 voxels, spacing 5, grid 16^3, phi ~ U[-2, 2] from seed 1: full volume."""
    shape, spacing = (64, 64, 64), (5, 5, 5)
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=1)
    assert phi.shape == (16, 16, 16, 3)
    got = gpu_forward(phi, shape, spacing)
    err, tol = fwd_err(got, phi, shape, spacing)
    assert err <= tol


# Volumes whose rows leave by tensor stores in blocks of rows (16-byte rows and
# strips; FP32 at x-spacings <= 4, BF16 with X % 8 == 0 -- at odd x-spacings in
# strips of 24 tiles): two to eight rows per block, ragged tails in x (a short
# last strip), y (a last tile-row inside the volume shorter than the block) and z.
TENSOR_STORE = [
    ((7, 13, 64), (2, 3, 1)),
    ((9, 22, 120), (3, 4, 2)),
    ((10, 17, 252), (4, 6, 3)),
    ((5, 30, 236), (2, 8, 4)),
    ((3, 12, 48), (1, 2, 4)),
    ((5, 30, 232), (2, 8, 4)),
    ((6, 20, 336), (3, 6, 6)),
    ((4, 17, 464), (2, 8, 8)),
    ((6, 23, 248), (2, 5, 5)),
    ((5, 14, 96), (3, 3, 3)),
]


@pytest.mark.parametrize("shape,spacing", TENSOR_STORE, ids=[f"{s}-{d}" for s, d in TENSOR_STORE])
def test_forward_tensor_store_blocks_match_oracle(shape, spacing):
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=7 + sum(shape) + sum(spacing))
    got = gpu_forward(phi, shape, spacing)
    err, tol = fwd_err(got, phi, shape, spacing)
    assert err <= tol, (err, tol)
    b16 = gpu_forward(phi, shape, spacing, dtype=torch.bfloat16)
    assert torch.equal(b16.cpu(), got.cpu().to(torch.bfloat16))


@pytest.mark.parametrize("shape,spacing", SMALL[:10], ids=[f"{s}-{d}" for s, d in SMALL[:10]])
def test_forward_bf16_is_rne_of_f32(shape, spacing):
    phi = synth.uniform_phi(shape, spacing, -4, 4, seed=3 + sum(shape))
    f32 = gpu_forward(phi, shape, spacing)
    b16 = gpu_forward(phi, shape, spacing, dtype=torch.bfloat16)
    # bit-exact: the BF16 field is round-to-nearest-even of the FP32 field
    assert torch.equal(b16.cpu(), f32.cpu().to(torch.bfloat16))
    want = oracle.forward(phi, shape, spacing)
    err = np.abs(b16.double().cpu().numpy() - want)
    bound = BF16_REL * np.abs(want) + FWD_TOL * np.max(np.abs(phi)) * (1 + BF16_REL)
    assert np.all(err <= bound)


def test_forward_unaligned_output_base():
    """Output rows start at every alignment mod 16 bytes (base offset by 1..3 floats)."""
    shape, spacing = (7, 9, 61), (3, 4, 5)
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=21)
    want = oracle.forward(phi, shape, spacing)
    n = int(np.prod(shape)) * 3
    for off in (1, 2, 3):
        buf = torch.full((n + 8,), 7.0, device=dev())
        out = buf[off:off + n].view(shape + (3,))
        gpu_forward(phi, shape, spacing, out=out)
        b = buf.cpu().numpy()
        assert np.all(b[:off] == 7.0) and np.all(b[off + n:] == 7.0), "wrote outside the output"
        assert np.max(np.abs(out.double().cpu().numpy() - want)) <= FWD_TOL * np.abs(phi).max()


@pytest.mark.parametrize("shape,spacing", SMALL, ids=[f"{s}-{d}" for s, d in SMALL])
def test_adjoint_matches_oracle(shape, spacing):
    rng = np.random.default_rng(sum(shape) * 7 + sum(spacing))
    g = rng.standard_normal(shape + (3,)).astype(np.float32)
    got = gpu_adjoint(g, spacing)
    err, tol = adj_err(got, g, spacing)
    assert err <= tol, (err, tol)


def test_adjoint_dot_product_identity_gpu():
    shape, spacing = (40, 37, 90), (5, 4, 6)
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=31)
    W = synth.normal_field(shape, seed=32)
    T = gpu_forward(phi, shape, spacing).double().cpu().numpy()
    A = gpu_adjoint(W, spacing).double().cpu().numpy()
    lhs, rhs = float(np.sum(T * W)), float(np.sum(phi.astype(np.float64) * A))
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1.0)


def test_adjoint_is_deterministic():
    shape, spacing = (50, 60, 70), (3, 4, 5)
    g = synth.normal_field(shape, seed=41)
    a = gpu_adjoint(g, spacing)
    b = gpu_adjoint(g, spacing)
    assert torch.equal(a, b)


# The adjoint's tensor-copy path (X % 4 == 0, dx <= 8, 16-byte-aligned
# gradient): every x-spacing, ragged y and z tails, dy = 8, several x-groups,
# X = 4 (a box wider than the array), blocks of 1, 4 and 5 rows
TMA = [
    ((9, 10, 12), (2, 2, 1)),
    ((11, 13, 40), (3, 5, 2)),
    ((7, 9, 96), (2, 7, 3)),
    ((10, 17, 116), (3, 8, 4)),
    ((12, 6, 160), (4, 3, 5)),
    ((5, 5, 244), (2, 2, 6)),
    ((6, 11, 212), (3, 4, 7)),
    ((9, 9, 264), (2, 2, 8)),
    ((20, 21, 4), (5, 5, 5)),
    ((9, 30, 40), (2, 10, 3)),      # dy = 10: blocks of 5 rows
    ((7, 25, 48), (3, 11, 4)),      # dy = 11 (prime): blocks of 1 row
    ((6, 35, 264), (2, 16, 8)),     # dx = 8, dy = 16: two boxes of 4 rows
    # y-spacings 4..6: units of two tile-rows (single-volume calls), odd and even
    # tile-row counts, several tile-plane chunks
    ((8, 40, 64), (2, 6, 4)),
    ((13, 24, 100), (5, 4, 3)),
    ((40, 18, 48), (3, 5, 4)),
]


@pytest.mark.parametrize("shape,spacing", TMA, ids=[f"{s}-{d}" for s, d in TMA])
def test_adjoint_tensor_copy_path_matches_oracle(shape, spacing):
    assert shape[2] % 4 == 0 and spacing[2] <= 8
    g = synth.normal_field(shape, seed=sum(shape) + 3 * sum(spacing))
    got = gpu_adjoint(g, spacing)
    err, tol = adj_err(got, g, spacing)
    assert err <= tol, (err, tol)


@pytest.mark.parametrize("shape,spacing", TMA[1::2], ids=[f"{s}-{d}" for s, d in TMA[1::2]])
def test_adjoint_tensor_copy_and_row_paths_agree(shape, spacing):
    """The same gradient 16-byte aligned (tensor-copy path) and 4 bytes off (row
    path).  With one tile-row per unit both paths add the same terms in the same
    order: bitwise equal.  A single volume at y-spacing 4..6 takes units of two
    tile-rows on the tensor-copy path, which sum a control point's terms in
    another order: there both results must match the oracle."""
    g_np = synth.normal_field(shape, seed=7 + sum(shape))
    g = torch.from_numpy(g_np).to(dev())
    n = g.numel()
    buf = torch.empty(n + 4, device=dev())
    assert buf.data_ptr() % 16 == 0
    off = buf[1:1 + n].view(g.shape)
    off.copy_(g)
    a = P.bsi_field_adjoint(g.contiguous(), spacing)
    b = P.bsi_field_adjoint(off, spacing)
    torch.cuda.synchronize()
    if 4 <= spacing[1] <= 6:
        for got in (a, b):
            err, tol = adj_err(got, g_np, spacing)
            assert err <= tol, (err, tol)
    else:
        assert torch.equal(a, b)


def test_empty_volumes():
    phi = torch.zeros(synth.grid_shape((0, 5, 5), (2, 2, 2)) + (3,), device=dev())
    out = P.bsi_field_forward(phi, (0, 5, 5), (2, 2, 2))
    assert out.shape == (0, 5, 5, 3)
    g = torch.zeros((4, 0, 6, 3), device=dev())
    d = P.bsi_field_adjoint(g, (2, 2, 2))
    torch.cuda.synchronize()
    assert d.shape == synth.grid_shape((4, 0, 6), (2, 2, 2)) + (3,)
    assert not d.any()


def test_adjoint_overwrites_output():
    shape, spacing = (10, 12, 14), (3, 3, 3)
    g = synth.normal_field(shape, seed=51)
    gt = torch.from_numpy(g).to(dev())
    out = torch.full(synth.grid_shape(shape, spacing) + (3,), 1e9, device=dev())
    ws = torch.full((P.bsi_adjoint_workspace_bytes(shape, spacing),), 255, dtype=torch.uint8, device=dev())
    P.bsi_field_adjoint(gt, spacing, out=out, workspace=ws)
    torch.cuda.synchronize()
    err, tol = adj_err(out, g, spacing)
    assert err <= tol


def test_batched_matches_per_volume_oracle():
    geoms = synth.batch_geometries(24, seed=55, xy_range=(8, 70), z_range=(8, 40), spacing_range=(1, 10))
    geoms.append(((0, 10, 10), (3, 3, 3)))
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    phis = [synth.uniform_phi(s, d, -3, 3, seed=100 + i) for i, (s, d) in enumerate(geoms)]
    grads = [synth.normal_field(s, seed=200 + i) for i, s in enumerate(shapes)]
    outs = P.bsi_field_forward_batched([torch.from_numpy(p).to(dev()) for p in phis], shapes, spacings)
    dphis = P.bsi_field_adjoint_batched([torch.from_numpy(g).to(dev()) for g in grads], spacings)
    torch.cuda.synchronize()
    for i, (s, d) in enumerate(geoms):
        err, tol = fwd_err(outs[i], phis[i], s, d)
        assert err <= tol, (i, s, d, err, tol)
        if np.prod(s) > 0:
            err, tol = adj_err(dphis[i], grads[i], d)
            assert err <= tol, (i, s, d, err, tol)
        else:
            assert not dphis[i].any()


def test_batched_more_than_one_launch_group():
    """More than 64 instances and a mix of specialised / generic x-spacings."""
    geoms = synth.batch_geometries(70, seed=57, xy_range=(5, 30), z_range=(5, 20), spacing_range=(2, 12))
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    phis = [synth.uniform_phi(s, d, -1, 1, seed=300 + i) for i, (s, d) in enumerate(geoms)]
    outs = P.bsi_field_forward_batched([torch.from_numpy(p).to(dev()) for p in phis], shapes, spacings)
    torch.cuda.synchronize()
    for i, (s, d) in enumerate(geoms):
        err, tol = fwd_err(outs[i], phis[i], s, d)
        assert err <= tol, (i, s, d)


def test_probe_fill_writes_the_pattern_exactly():
    """bsi_probe_fill (the write-peak probe): every byte of [dst, dst + bytes)
    holds the pattern and nothing after it is touched, for whole 16 KB chunks
    plus a tail."""
    for nbytes in (16, 16 * 1024, 5 * 16 * 1024 + 48, 3 << 20):
        buf = torch.zeros(nbytes // 4 + 8, dtype=torch.int32, device=dev())
        P.bsi_probe_fill(buf[: nbytes // 4], 0x01020304)
        torch.cuda.synchronize()
        assert bool((buf[: nbytes // 4] == 0x01020304).all()), nbytes
        assert bool((buf[nbytes // 4:] == 0).all()), nbytes
