"""Scalar (one-channel) BSI -- image interpolation / zooming with the image
samples as control points -- CUDA path vs the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import BF16_REL, FWD_TOL, dev

pytestmark = pytest.mark.gpu

CASES = [
    ((64, 64, 64), (5, 5, 5)),
    ((14, 21, 236), (3, 5, 4)),     # x-spacing 4, X % 4 == 0: direct 16-byte stores, 3 strips
    ((9, 10, 11), (2, 2, 2)),
    ((13, 7, 40), (3, 2, 3)),
    ((17, 19, 23), (4, 4, 4)),
    ((20, 11, 93), (6, 5, 5)),
    ((12, 13, 100), (5, 6, 6)),
    ((15, 9, 97), (7, 3, 7)),
    ((16, 16, 250), (8, 8, 8)),
    ((11, 12, 300), (4, 3, 9)),      # generic x-spacing
    ((1, 1, 1), (1, 1, 1)),
    ((33, 1, 1), (5, 1, 1)),
]


def _oracle_scalar(coeff, shape, spacing):
    """Eq. 1 for one channel: the (pinned) 3-channel oracle with the grid in channel 0."""
    phi = np.zeros(coeff.shape + (3,), np.float64)
    phi[..., 0] = coeff
    return oracle.forward(phi, shape, spacing)[..., 0]


@pytest.mark.parametrize("shape,spacing", CASES, ids=[f"{s}-{d}" for s, d in CASES])
def test_scalar_forward_matches_oracle(shape, spacing):
    rng = np.random.default_rng(sum(shape) + 5 * sum(spacing))
    coeff = rng.uniform(-2, 2, synth.grid_shape(shape, spacing)).astype(np.float32)
    got = P.bsi_scalar_forward(torch.from_numpy(coeff).to(dev()), shape, spacing)
    torch.cuda.synchronize()
    want = _oracle_scalar(coeff, shape, spacing)
    err = float(np.max(np.abs(got.double().cpu().numpy() - want)))
    assert err <= FWD_TOL * float(np.max(np.abs(coeff))), err


@pytest.mark.parametrize("shape,spacing", CASES[:8], ids=[f"{s}-{d}" for s, d in CASES[:8]])
def test_scalar_is_channel_of_the_field_bitwise(shape, spacing):
    """One channel computed alone equals that channel of the 3-channel field bit
    for bit (same weights, same FMA order), for FP32 and BF16 output."""
    rng = np.random.default_rng(3 + sum(shape))
    phi = rng.uniform(-3, 3, synth.grid_shape(shape, spacing) + (3,)).astype(np.float32)
    phit = torch.from_numpy(phi).to(dev())
    for dt in (torch.float32, torch.bfloat16):
        field = P.bsi_field_forward(phit, shape, spacing, out_dtype=dt)
        for c in range(3):
            s = P.bsi_scalar_forward(phit[..., c].contiguous(), shape, spacing, out_dtype=dt)
            torch.cuda.synchronize()
            assert torch.equal(s, field[..., c]), (dt, c)


# One-channel volumes whose rows leave by tensor stores in blocks of rows (FP32 at
# x-spacings <= 3, BF16 at even x-spacings with X % 8 == 0): block heights 3..8,
# ragged tails in x, y and z.
TENSOR_STORE = [
    ((7, 30, 64), (2, 6, 2)),
    ((9, 22, 120), (3, 4, 4)),
    ((5, 18, 336), (2, 3, 6)),
    ((4, 17, 464), (2, 8, 8)),
]


@pytest.mark.parametrize("shape,spacing", TENSOR_STORE, ids=[f"{s}-{d}" for s, d in TENSOR_STORE])
def test_scalar_tensor_store_blocks(shape, spacing):
    """Against the oracle (FP32), BF16 against round-to-nearest-even of FP32, and
    each against the same channel of the 3-channel field, bit for bit."""
    rng = np.random.default_rng(11 + sum(shape))
    phi = rng.uniform(-3, 3, synth.grid_shape(shape, spacing) + (3,)).astype(np.float32)
    phit = torch.from_numpy(phi).to(dev())
    coeff = phit[..., 1].contiguous()
    f32 = P.bsi_scalar_forward(coeff, shape, spacing)
    b16 = P.bsi_scalar_forward(coeff, shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    want = _oracle_scalar(phi[..., 1], shape, spacing)
    err = float(np.max(np.abs(f32.double().cpu().numpy() - want)))
    assert err <= FWD_TOL * float(np.max(np.abs(phi[..., 1]))), err
    assert torch.equal(b16.cpu(), f32.cpu().to(torch.bfloat16))
    for dt, got in ((torch.float32, f32), (torch.bfloat16, b16)):
        field = P.bsi_field_forward(phit, shape, spacing, out_dtype=dt)
        torch.cuda.synchronize()
        assert torch.equal(got, field[..., 1]), dt


def test_scalar_direct_stores_equal_the_staged_path():
    """At x-spacing 4 with rows on 16-byte boundaries each lane stores its tile
    as one 16-byte vector; an output 4 bytes off that boundary takes the staged
    bulk-copy path.  Both give the same bits."""
    shape, spacing = (10, 13, 120), (4, 3, 4)
    rng = np.random.default_rng(41)
    coeff = torch.from_numpy(rng.uniform(-2, 2, synth.grid_shape(shape, spacing)).astype(np.float32)).to(dev())
    n = shape[0] * shape[1] * shape[2]
    buf = torch.empty(n + 4, device=dev())
    aligned = P.bsi_scalar_forward(coeff, shape, spacing)
    assert aligned.data_ptr() % 16 == 0
    off = buf[1:n + 1].view(shape)
    assert off.data_ptr() % 16 == 4
    P.bsi_scalar_forward(coeff, shape, spacing, out=off)
    torch.cuda.synchronize()
    assert torch.equal(aligned, off)
    assert P.bsi_check_device_status() == 0


def test_scalar_zoom_of_a_smooth_image():
    """Zooming: an image's samples as the control points at spacing 4 (a 4x
    zoom of a 30 x 40 x 50 image, one border sample per side); the result stays
    within the FP32 tolerance of the oracle and keeps the image's range (B-spline
    weights are a partition of unity)."""
    img = synth.blob_image((30 + 3, 40 + 3, 50 + 3), seed=8)      # grid dims ceil(N/4) + 3
    shape, spacing = (30 * 4, 40 * 4, 50 * 4), (4, 4, 4)
    assert img.shape == synth.grid_shape(shape, spacing)
    z = P.bsi_scalar_forward(torch.from_numpy(img).to(dev()), shape, spacing)
    bf = P.bsi_scalar_forward(torch.from_numpy(img).to(dev()), shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    zc = z.double().cpu().numpy()
    assert zc.min() >= float(img.min()) - 1e-5 and zc.max() <= float(img.max()) + 1e-5
    pts = synth.sample_voxels(shape, 400, seed=9)
    phi = np.zeros(img.shape + (3,), np.float64)
    phi[..., 0] = img
    want = oracle.forward_points(phi, shape, spacing, pts)[:, 0]
    got = zc[pts[:, 2], pts[:, 1], pts[:, 0]]
    assert float(np.max(np.abs(got - want))) <= FWD_TOL * float(np.max(np.abs(img)))
    ref16 = z.to(torch.bfloat16)
    assert torch.equal(bf, ref16)
