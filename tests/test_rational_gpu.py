"""Non-integer, non-aligned spacing (bsi_field_forward_rational) against the
FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import ADJ_TOL, FWD_TOL, dev

pytestmark = pytest.mark.gpu

# (shape (Z, Y, X), num, den, off), each (z, y, x): spacing num/den, lattice shift off/den.
# x-spacing 4..8 with mostly full 29-cell strips runs the strip kernel (z-cells
# split into parts when the volume has few cells); other volumes the windowed
# kernel (nx <= 1024) or the row-per-warp kernel.
CASES = [
    ((13, 17, 50), (5, 7, 9), (2, 2, 2), (0, 3, 1)),           # 2.5, 3.5, 4.5
    ((12, 20, 64), (4, 3, 10), (3, 1, 3), (2, 0, 7)),          # 1.33, 3, 3.33
    ((9, 11, 40), (1, 9, 7), (1, 4, 5), (0, 8, 6)),            # 1, 2.25, 1.4
    ((20, 16, 70), (47, 47, 47), (10, 10, 10), (3, 0, 9)),     # 4.7 (a CT voxel ratio), shifted
    ((9, 10, 136), (47, 47, 47), (10, 10, 10), (3, 0, 9)),     # 4.7, one full strip: strip kernel, z-cells split
    ((8, 9, 100), (5, 5, 5), (1, 1, 1), (0, 0, 0)),            # integer spacing on this path
    ((10, 10, 33), (640, 13, 23), (10, 5, 7), (639, 4, 22)),   # spacing 64; shift near a full cell
    ((1, 1, 1), (3, 3, 3), (2, 2, 2), (1, 1, 1)),
    ((3, 5, 1100), (2, 3, 1), (1, 2, 1), (1, 1, 0)),          # nx = 1103: the row-per-warp kernel
    ((40, 37, 30), (7, 9, 11), (3, 4, 5), (2, 5, 10)),         # several 16-row runs per plane
    ((3, 4, 2500), (5, 5, 47), (2, 2, 10), (1, 0, 7)),         # X > 2048: x weights computed per voxel
    ((6, 7, 464), (3, 5, 8), (1, 2, 1), (0, 4, 0)),            # x-spacing 8: full 232-voxel segments
    ((30, 41, 97), (13, 11, 17), (2, 2, 4), (1, 0, 3)),        # 4.25: one strip, several y- and z-cells
    ((10, 12, 200), (3, 5, 47), (1, 2, 5), (0, 1, 3)),         # 9.4: windowed kernel
    ((40, 37, 30), (7, 9, 55), (3, 4, 5), (2, 5, 10)),         # 11: windowed, several runs per plane
    ((2, 3, 10000), (2, 3, 47), (1, 1, 5), (1, 0, 2)),         # nx = 1067: the row-per-warp kernel
]


@pytest.mark.parametrize("shape,num,den,off", CASES, ids=[f"{c[0]}-{c[1]}/{c[2]}+{c[3]}" for c in CASES])
def test_rational_forward_matches_oracle(shape, num, den, off):
    grid = P.rational_grid_shape(shape, num, den, off)
    rng = np.random.default_rng(sum(shape) + sum(num))
    phi = rng.uniform(-3, 3, grid + (3,)).astype(np.float32)
    got = P.bsi_field_forward_rational(torch.from_numpy(phi).to(dev()), shape, num, den, off)
    torch.cuda.synchronize()
    want = oracle.forward_rational(phi, shape, num, den, off)
    err = float(np.max(np.abs(got.double().cpu().numpy() - want)))
    assert err <= FWD_TOL * float(np.max(np.abs(phi))), err
    assert P.bsi_check_device_status() == 0


def test_rational_with_integer_spacing_matches_the_strip_kernel():
    """den = 1, off = 0: the same field as bsi_field_forward (weights computed
    per voxel in FP32 instead of tabulated in FP64: within the FP32 tolerance)."""
    shape, spacing = (30, 40, 90), (3, 4, 5)
    phi = torch.from_numpy(synth.uniform_phi(shape, spacing, -2, 2, seed=77)).to(dev())
    a = P.bsi_field_forward(phi, shape, spacing)
    b = P.bsi_field_forward_rational(phi, shape, spacing, (1, 1, 1), (0, 0, 0))
    torch.cuda.synchronize()
    assert float((a - b).abs().max()) <= 2 * FWD_TOL * 2.0


@pytest.mark.parametrize("shape,num,den,off", CASES, ids=[f"{c[0]}-{c[1]}/{c[2]}+{c[3]}" for c in CASES])
def test_rational_adjoint_matches_oracle(shape, num, den, off):
    """Transpose of the non-integer-spacing forward against the FP64 scatter
    oracle, element by element over the whole grid."""
    rng = np.random.default_rng(3 * sum(shape) + sum(den))
    G = rng.standard_normal(shape + (3,)).astype(np.float32)
    got = P.bsi_field_adjoint_rational(torch.from_numpy(G).to(dev()), num, den, off)
    torch.cuda.synchronize()
    want = oracle.adjoint_rational(G, num, den, off)
    assert got.shape == want.shape
    err = float(np.max(np.abs(got.double().cpu().numpy() - want)))
    assert err <= ADJ_TOL * max(float(np.max(np.abs(want))), 1e-30), err
    assert P.bsi_check_device_status() == 0


def test_rational_adjoint_is_the_transpose_and_deterministic():
    """<forward(phi), G> = <phi, adjoint(G)> on the GPU (FP32 sums, relative
    1e-5), and two adjoint calls give the same bits."""
    shape, num, den, off = (30, 41, 97), (13, 11, 17), (2, 2, 4), (1, 0, 3)
    rng = np.random.default_rng(71)
    phi = torch.from_numpy(rng.uniform(-2, 2, P.rational_grid_shape(shape, num, den, off) + (3,))
                           .astype(np.float32)).to(dev())
    G = torch.from_numpy(rng.standard_normal(shape + (3,)).astype(np.float32)).to(dev())
    T = P.bsi_field_forward_rational(phi, shape, num, den, off)
    a = P.bsi_field_adjoint_rational(G, num, den, off)
    b = P.bsi_field_adjoint_rational(G, num, den, off)
    torch.cuda.synchronize()
    lhs = float((T.double() * G.double()).sum())
    rhs = float((phi.double() * a.double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * max(abs(lhs), 1.0)
    assert torch.equal(a, b)


def test_rational_adjoint_of_an_empty_volume_is_zero():
    shape, num, den, off = (0, 5, 7), (5, 5, 5), (2, 2, 2), (0, 0, 0)
    G = torch.empty(shape + (3,), device=dev())
    out = torch.full(P.rational_grid_shape(shape, num, den, off) + (3,), 7.0, device=dev())
    P.bsi_field_adjoint_rational(G, num, den, off, out=out)
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0


def test_field_rational_autograd_uses_the_adjoint():
    """field_rational's backward is bsi_field_adjoint_rational, bit for bit."""
    shape, num, den, off = (20, 16, 70), (47, 47, 47), (10, 10, 10), (3, 0, 9)
    rng = np.random.default_rng(72)
    phi = torch.from_numpy(rng.uniform(-2, 2, P.rational_grid_shape(shape, num, den, off) + (3,))
                           .astype(np.float32)).to(dev()).requires_grad_()
    W = torch.from_numpy(rng.standard_normal(shape + (3,)).astype(np.float32)).to(dev())
    (P.field_rational(phi, shape, num, den, off) * W).sum().backward()
    want = P.bsi_field_adjoint_rational(W, num, den, off)
    torch.cuda.synchronize()
    assert torch.equal(phi.grad, want)
