"""Full-size workloads (the sizes and launch configuration the benchmark times),
checked against the FP64 oracle at EVERY voxel and EVERY control point.

The forward is compared with Eq. 1 (Sec. 2.1) evaluated by the oracle voxel
by voxel, a chunk of z-planes at a time; the adjoint with the oracle's
transpose of Eq. 1 over the whole grid.  Tolerances: forward
max|err| <= 1e-5 max|phi|, adjoint max|err| <= 1e-5 max|oracle dphi|, BF16
|err| <= 2^-8 |T| + (1 + 2^-8) 1e-5 max|phi| (round to nearest even of the
FP32 result).
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import (ADJ_TOL, BF16_REL, FWD_TOL, FieldError, dev, full_adjoint_check, full_forward_check,
                      host_planes, oracle_by_planes, plane_points)

pytestmark = pytest.mark.gpu

CT = ((300, 512, 512), (5, 5, 5))
SWEEP = [(3, 3, 3), (5, 5, 5), (6, 5, 4), (8, 8, 8)]
BIG = (512, 512, 512)


def grid_points(grid):
    """Every stored control point of a grid (nz, ny, nx) as (gx, gy, gz) rows."""
    nz, ny, nx = grid
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int64)


def test_ct_forward_f32_and_bf16_full():
    """CT-shaped 512 x 512 x 300 at spacing 5: FP32 and BF16 fields at every voxel."""
    shape, spacing = CT
    phi = synth.gaussian_random_phi(shape, spacing, sigma_vox=3.0, smooth_cells=2.0, seed=2)
    assert phi.shape == (63, 106, 106, 3)
    t = torch.from_numpy(phi).to(dev())
    out = P.bsi_field_forward(t, shape, spacing)
    b16 = P.bsi_field_forward(t, shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    # BF16 is the RNE rounding of the FP32 field, bit for bit, everywhere
    assert torch.equal(b16, out.to(torch.bfloat16))
    atol = FWD_TOL * float(np.abs(phi).max())
    errs = full_forward_check(phi, shape, spacing, {
        "f32": (out, FieldError(atol)),
        "bf16": (b16, FieldError((1 + BF16_REL) * atol, rel=BF16_REL)),
    })
    assert errs["f32"][1].ok, errs["f32"][1]
    assert errs["bf16"][1].ok, errs["bf16"][1]


def test_ct_adjoint_full():
    shape, spacing = CT
    g = synth.normal_field(shape, seed=4)
    d = P.bsi_field_adjoint(torch.from_numpy(g).to(dev()), spacing)
    torch.cuda.synchronize()
    err = full_adjoint_check(g, spacing, d)
    assert err.ok, err


@pytest.mark.parametrize("spacing", SWEEP)
def test_512cubed_sweep_forward_full(spacing):
    phi = synth.uniform_phi(BIG, spacing, -4, 4, seed=3)
    out = torch.full(BIG + (3,), float("nan"), device=dev())   # every voxel must be written
    P.bsi_field_forward(torch.from_numpy(phi).to(dev()), BIG, spacing, out=out)
    torch.cuda.synchronize()
    errs = full_forward_check(phi, BIG, spacing, {"f32": (out, FieldError(FWD_TOL * float(np.abs(phi).max())))})
    assert errs["f32"][1].ok, errs["f32"][1]


@pytest.mark.parametrize("spacing", SWEEP)
def test_512cubed_sweep_adjoint_full(spacing):
    g = synth.normal_field(BIG, seed=30 + sum(spacing))
    d = torch.full(synth.grid_shape(BIG, spacing) + (3,), float("nan"), device=dev())
    P.bsi_field_adjoint(torch.from_numpy(g).to(dev()), spacing, out=d)
    torch.cuda.synchronize()
    err = full_adjoint_check(g, spacing, d)
    assert err.ok, err


def test_batched_64_instances_full():
    """The 64-volume uneven batch: every volume's field and dL/dphi in full."""
    geoms = synth.batch_geometries(64, seed=5)
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    total = sum(int(np.prod(s)) for s in shapes)
    assert 1.0e8 < total < 2.5e8
    phis = [synth.uniform_phi(s, d, -3, 3, seed=500 + i) for i, (s, d) in enumerate(geoms)]
    outs = P.bsi_field_forward_batched([torch.from_numpy(p).to(dev()) for p in phis], shapes, spacings)
    grads = [synth.normal_field(shapes[i], seed=600 + i) for i in range(64)]
    dphis = P.bsi_field_adjoint_batched([torch.from_numpy(g).to(dev()) for g in grads], spacings)
    torch.cuda.synchronize()
    for i in range(64):
        errs = full_forward_check(phis[i], shapes[i], spacings[i],
                                  {"f32": (outs[i], FieldError(FWD_TOL * float(np.abs(phis[i]).max())))},
                                  planes=64)
        assert errs["f32"][1].ok, (i, shapes[i], spacings[i], errs["f32"][1])
        err = full_adjoint_check(grads[i], spacings[i], dphis[i])
        assert err.ok, (i, shapes[i], spacings[i], err)


def _lipschitz(F):
    L = sum(float(np.max(np.abs(np.diff(F.astype(np.float64), axis=ax)))) for ax in range(3) if F.shape[ax] > 1)
    return L + float(np.max(np.abs(F)))


def test_ct_resample_forward_and_backward_full():
    """The bench's resampling workload (CT control grid, 8-blob floating image):
    warped values at every voxel; dL/dphi at every control point against the
    oracle's chain (interpolant gradient at x + T(x), times dL/dwarped,
    transposed through Eq. 1).

    The trilinear interpolant's gradient jumps where a sample position crosses
    an integer, so a voxel whose position lies within FP32 rounding of one may
    take either side.  dL/dwarped is set to zero at the voxels whose oracle
    position lies within 1e-4 voxels of an integer on any axis (about 0.06% of
    them), on both sides; everywhere else both sides sample inside the same
    cell and the chain is smooth."""
    shape, spacing = CT
    Z, Y, X = shape
    phi = synth.gaussian_random_phi(shape, spacing, sigma_vox=3.0, smooth_cells=2.0, seed=2)
    F = synth.blob_image(shape, seed=6)
    pt, Ft = torch.from_numpy(phi).to(dev()), torch.from_numpy(F).to(dev())
    W = P.bsi_resample_forward(pt, shape, spacing, Ft)
    torch.cuda.synchronize()
    # values: a position error of e voxels moves a trilinear sample by at most
    # e times the interpolant's Lipschitz bound
    tol = 1e-5 * float(np.max(np.abs(phi))) * _lipschitz(F) + 1e-6 * float(np.max(np.abs(F)))
    err = FieldError(tol)
    fn = lambda pts: oracle.resample_points(phi, shape, spacing, F, pts)[0]
    for z0, z1, want in oracle_by_planes(fn, shape, planes=32, threaded=True):
        err.add(host_planes(W, z0, z1, (Y, X, 1)), want)
    assert err.ok, err

    dW = np.random.default_rng(5).standard_normal(shape, dtype=np.float32)
    fn = lambda pts: oracle.forward_points(phi, shape, spacing, pts)
    kinks = 0
    for z0, z1, T in oracle_by_planes(fn, shape, planes=32):
        pos = plane_points(Y, X, z0, z1).reshape(z1 - z0, Y, X, 3) + T   # (x, y, z) + T
        fr = pos - np.floor(pos)
        near = (np.minimum(fr, 1.0 - fr) < 1e-4).any(axis=-1)
        dW[z0:z1][near] = 0.0
        kinks += int(near.sum())
    assert 0 < kinks < 2e-3 * dW.size
    dphi = P.bsi_resample_backward(pt, shape, spacing, Ft, torch.from_numpy(dW).to(dev()))
    torch.cuda.synchronize()
    want = oracle.resample_backward(phi, shape, spacing, F, dW)
    derr = FieldError(ADJ_TOL * float(np.max(np.abs(want))))
    derr.add(dphi.double().cpu().numpy(), want)
    assert derr.ok, derr


def test_ct_rational_forward_full():
    """The bench's non-integer spacing workload: 512x512x300 at 4.7 voxels with
    the lattice shifted by (0.3, 0, 0.9) (z, y, x)."""
    shape, num, den, off = (300, 512, 512), (47, 47, 47), (10, 10, 10), (3, 0, 9)
    grid = P.rational_grid_shape(shape, num, den, off)
    phi = np.random.default_rng(9).uniform(-3, 3, grid + (3,)).astype(np.float32)
    out = P.bsi_field_forward_rational(torch.from_numpy(phi).to(dev()), shape, num, den, off)
    torch.cuda.synchronize()
    err = FieldError(FWD_TOL * float(np.max(np.abs(phi))))
    fn = lambda pts: oracle.forward_rational_points(phi, shape, num, den, off, pts)
    Z, Y, X = shape
    for z0, z1, want in oracle_by_planes(fn, shape, planes=32, threaded=True):
        err.add(host_planes(out, z0, z1, (Y, X, 3)), want)
    assert err.ok, err


def test_ct_rational_adjoint_full():
    """The adjoint of the non-integer spacing workload (512x512x300 at 4.7
    voxels, shifted lattice) at every control point."""
    shape, num, den, off = (300, 512, 512), (47, 47, 47), (10, 10, 10), (3, 0, 9)
    G = synth.normal_field(shape, seed=10)
    dphi = P.bsi_field_adjoint_rational(torch.from_numpy(G).to(dev()), num, den, off)
    torch.cuda.synchronize()
    gpts = grid_points(P.rational_grid_shape(shape, num, den, off))
    nt = oracle.threads()
    with ThreadPoolExecutor(nt) as pool:
        parts = pool.map(lambda q: oracle.adjoint_rational_points(G, num, den, off, q), np.array_split(gpts, 4 * nt))
        want = np.concatenate(list(parts)).reshape(dphi.shape)
    err = FieldError(ADJ_TOL * float(np.max(np.abs(want))))
    err.add(dphi.double().cpu().numpy(), want)
    assert err.ok, err


def test_ct_scalar_zoom_full():
    """The bench's scalar workload: a 4x zoom of a 128 x 128 x 75 image (plus
    border) to 512 x 512 x 300, FP32 and BF16, at every voxel."""
    shape, spacing = (300, 512, 512), (4, 4, 4)
    img = synth.blob_image(synth.grid_shape(shape, spacing), seed=7)
    t = torch.from_numpy(img).to(dev())
    z = P.bsi_scalar_forward(t, shape, spacing)
    zb = P.bsi_scalar_forward(t, shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    assert torch.equal(zb, z.to(torch.bfloat16))
    # one channel of Eq. 1 does not see the others: the image in channel 0
    phi = np.zeros(img.shape + (3,), np.float64)
    phi[..., 0] = img
    err = FieldError(FWD_TOL * float(np.max(np.abs(img))))
    fn = lambda pts: oracle.forward_points(phi, shape, spacing, pts)[:, :1]
    Z, Y, X = shape
    for z0, z1, want in oracle_by_planes(fn, shape, planes=32):
        err.add(host_planes(z, z0, z1, (Y, X, 1)), want)
    assert err.ok, err
