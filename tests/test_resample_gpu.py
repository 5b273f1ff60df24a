"""BSI fused with the resampling of a floating image (bsi_resample_*), CUDA
path vs the FP64 oracle, element by element, through the C ABI."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import ADJ_TOL, dev

pytestmark = pytest.mark.gpu

# (volume (Z, Y, X), spacing (dz, dy, dx), floating image (fZ, fY, fX), displacement amplitude)
CASES = [
    ((24, 20, 40), (5, 5, 5), (24, 20, 40), 3.0),
    ((13, 17, 29), (2, 3, 1), (15, 12, 31), 2.0),      # image of another size
    ((9, 30, 64), (3, 4, 4), (9, 30, 64), 6.0),        # many samples outside the image
    ((11, 10, 100), (4, 2, 8), (11, 10, 100), 2.5),    # 16-byte vector path of the forward (dx = 8)
    ((10, 12, 61), (3, 3, 6), (10, 12, 61), 2.0),
    ((7, 9, 130), (2, 3, 7), (8, 9, 128), 1.5),        # several x-groups
    ((8, 9, 140), (3, 5, 13), (8, 9, 140), 2.0),       # generic x-spacing
    ((1, 1, 3), (1, 1, 1), (2, 2, 2), 1.0),
    ((30, 1, 1), (5, 1, 1), (30, 1, 1), 4.0),       # floating image 1 voxel wide and high
    ((12, 10, 16), (3, 2, 4), (12, 10, 2), 3.0),    # floating image 2 voxels wide
]


def _image(shape, seed):
    """Smooth image: a sum of Gaussian blobs (the registration images' stand-in)."""
    return synth.blob_image(shape, seed=seed).astype(np.float32)


def _lipschitz(F):
    """Sum over axes of the largest neighbour difference: |F~(p) - F~(q)| <= L |p - q|_inf."""
    L = 0.0
    for ax in range(3):
        if F.shape[ax] > 1:
            L += float(np.max(np.abs(np.diff(F.astype(np.float64), axis=ax))))
    return L + float(np.max(np.abs(F)))   # the zero extension adds a step of up to max|F|


def _run(shape, spacing, fshape, amp, seed):
    phi = synth.uniform_phi(shape, spacing, -amp, amp, seed=seed)
    F = _image(fshape, seed + 1)
    W = P.bsi_resample_forward(torch.from_numpy(phi).to(dev()), shape, spacing, torch.from_numpy(F).to(dev()))
    torch.cuda.synchronize()
    return phi, F, W.double().cpu().numpy()


@pytest.mark.parametrize("shape,spacing,fshape,amp", CASES, ids=[f"{c[0]}-{c[1]}" for c in CASES])
def test_resample_forward_matches_oracle(shape, spacing, fshape, amp):
    phi, F, W = _run(shape, spacing, fshape, amp, seed=sum(shape) + 7 * sum(spacing))
    want = oracle.resample(phi, shape, spacing, F)
    # position error <= the forward's 1e-5 max|phi| bound; the interpolant moves
    # at most L per voxel of position; plus FP32 rounding of the 7 lerps
    tol = 1e-5 * max(float(np.max(np.abs(phi))), 1.0) * _lipschitz(F) + 1e-6 * float(np.max(np.abs(F)))
    err = float(np.max(np.abs(W - want)))
    assert err <= tol, (err, tol)


def test_resample_identity_and_integer_shift_are_exact():
    shape, spacing = (12, 14, 40), (3, 4, 5)
    F = _image(shape, 3)
    Ft = torch.from_numpy(F).to(dev())
    phi = torch.zeros(synth.grid_shape(shape, spacing) + (3,), device=dev())
    W = P.bsi_resample_forward(phi, shape, spacing, Ft)
    torch.cuda.synchronize()
    assert torch.equal(W, Ft)
    phi = torch.full(synth.grid_shape(shape, spacing) + (3,), 0.0, device=dev())
    phi[..., 0], phi[..., 1], phi[..., 2] = 2.0, -1.0, 3.0
    W = P.bsi_resample_forward(phi, shape, spacing, Ft).double().cpu().numpy()
    want = oracle.resample(phi.cpu().numpy(), shape, spacing, F)
    assert float(np.max(np.abs(W - want))) <= 1e-6 * float(np.max(np.abs(F)))


def _kink_free(phi, shape, spacing, eps=1e-4):
    """Voxels whose sample position is at least eps from an integer in every axis
    (the interpolant's gradient jumps at integers)."""
    T = oracle.forward(phi, shape, spacing)
    Z, Y, X = shape
    z, y, x = np.meshgrid(np.arange(Z), np.arange(Y), np.arange(X), indexing="ij")
    ok = np.ones(shape, bool)
    for q in (x + T[..., 0], y + T[..., 1], z + T[..., 2]):
        f = q - np.floor(q)
        ok &= (f > eps) & (f < 1 - eps)
    return ok


# the backward's cases: the first seven above, plus strips side by side (their
# partial sums overlap by 3-4 columns) and several chunks of tile-planes
BWD_CASES = CASES[:7] + [
    ((6, 7, 300), (2, 3, 3), (6, 7, 300), 2.0),      # 4 strips of the forward's tiles
    ((26, 9, 120), (2, 4, 5), (26, 9, 120), 2.5),    # 4 chunks of tile-planes, 1 strip
]


@pytest.mark.parametrize("shape,spacing,fshape,amp", BWD_CASES, ids=[f"{c[0]}-{c[1]}" for c in BWD_CASES])
def test_resample_backward_matches_oracle(shape, spacing, fshape, amp):
    """dL/dphi vs the oracle's chain (interpolant gradient at x + T(x), times
    dL/dwarped, transposed through Eq. 1).  The interpolant's gradient jumps
    where a sample position crosses an integer, so dL/dwarped is set to zero
    at the voxels whose position lies within 1e-4 of an integer on any axis, on
    both sides."""
    seed = sum(shape) + 11 * sum(spacing)
    phi = synth.uniform_phi(shape, spacing, -amp, amp, seed=seed)
    F = _image(fshape, seed + 1)
    dW = synth.normal_field(shape, seed=seed + 2)[..., 0].copy()
    dW[~_kink_free(phi, shape, spacing)] = 0.0
    phit, Ft, dWt = (torch.from_numpy(a).to(dev()) for a in (phi, F, dW))
    nbytes = P.bsi_resample_backward_workspace_bytes(shape, spacing)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev())
    got = P.bsi_resample_backward(phit, shape, spacing, Ft, dWt, workspace=ws)
    again = P.bsi_resample_backward(phit, shape, spacing, Ft, dWt)
    torch.cuda.synchronize()
    assert torch.equal(got, again)   # deterministic: fixed-order reduce, no atomics
    want = oracle.resample_backward(phi, shape, spacing, F, dW)
    err = float(np.max(np.abs(got.double().cpu().numpy() - want)))
    assert err <= ADJ_TOL * max(float(np.max(np.abs(want))), 1e-30), err


def test_resample_autograd_matches_entry_points():
    shape, spacing = (16, 18, 44), (4, 3, 5)
    phi = torch.from_numpy(synth.uniform_phi(shape, spacing, -2, 2, seed=61)).to(dev()).requires_grad_(True)
    F = torch.from_numpy(_image(shape, 62)).to(dev())
    w = torch.from_numpy(synth.normal_field(shape, seed=63)[..., 0].copy()).to(dev())
    W = P.resample(phi, F, shape, spacing)
    (W * w).sum().backward()
    with torch.no_grad():
        W2 = P.bsi_resample_forward(phi.detach(), shape, spacing, F)
        g2 = P.bsi_resample_backward(phi.detach(), shape, spacing, F, w)
    torch.cuda.synchronize()
    assert torch.equal(W, W2)
    assert torch.equal(phi.grad, g2)


def test_resample_validation():
    shape, spacing = (4, 5, 6), (2, 2, 2)
    phi = torch.zeros(synth.grid_shape(shape, spacing) + (3,), device=dev())
    F = torch.zeros((4, 5, 6), device=dev())
    with pytest.raises(Exception):
        P.bsi_resample_forward(phi, shape, spacing, torch.zeros((0, 5, 6), device=dev()))
    out = P.bsi_resample_forward(phi, shape, spacing, F)
    torch.cuda.synchronize()
    assert not out.any()
    assert P.bsi_check_device_status() == 0
