"""Full-size workloads (the sizes and launch configuration the benchmark times),
checked on sampled outputs the oracle computes one by one."""
import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import ADJ_TOL, BF16_REL, FWD_TOL, dev

pytestmark = pytest.mark.gpu

CT = ((300, 512, 512), (5, 5, 5))


def _sampled_fwd(phi, shape, spacing, out, npts=3000, seed=0):
    pts = synth.sample_voxels(shape, npts, seed)
    want = oracle.forward_points(phi, shape, spacing, pts)
    idx = torch.from_numpy(pts).to(out.device)
    got = out[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    return got, want


def test_ct_forward_f32_and_bf16_sampled():
    shape, spacing = CT
    phi = synth.gaussian_random_phi(shape, spacing, sigma_vox=3.0, smooth_cells=2.0, seed=2)
    assert phi.shape == (63, 106, 106, 3)
    t = torch.from_numpy(phi).to(dev())
    out = P.bsi_field_forward(t, shape, spacing)
    torch.cuda.synchronize()
    got, want = _sampled_fwd(phi, shape, spacing, out, seed=2)
    assert np.max(np.abs(got - want)) <= FWD_TOL * np.abs(phi).max()
    b16 = P.bsi_field_forward(t, shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    # BF16 is the RNE rounding of the FP32 field (bit-exact on one z-slab per 50)
    for z in range(0, shape[0], 50):
        assert torch.equal(b16[z], out[z].to(torch.bfloat16))
    gb, _ = _sampled_fwd(phi, shape, spacing, b16, seed=2)
    assert np.all(np.abs(gb - want) <= BF16_REL * np.abs(want) + FWD_TOL * np.abs(phi).max() * 1.01)


@pytest.mark.parametrize("spacing", [(3, 3, 3), (5, 5, 5), (6, 5, 4), (8, 8, 8)])
def test_512cubed_sweep_forward_sampled(spacing):
    shape = (512, 512, 512)
    phi = synth.uniform_phi(shape, spacing, -4, 4, seed=3)
    out = P.bsi_field_forward(torch.from_numpy(phi).to(dev()), shape, spacing)
    torch.cuda.synchronize()
    got, want = _sampled_fwd(phi, shape, spacing, out, seed=sum(spacing))
    assert np.max(np.abs(got - want)) <= FWD_TOL * np.abs(phi).max()
    # every value written and finite (the buffer starts as NaN)
    out2 = torch.full_like(out, float("nan"))
    P.bsi_field_forward(torch.from_numpy(phi).to(dev()), shape, spacing, out=out2)
    torch.cuda.synchronize()
    assert bool(torch.isfinite(out2).all())
    assert torch.equal(out, out2)


def test_ct_adjoint_sampled():
    shape, spacing = CT
    g = synth.normal_field(shape, seed=4)
    d = P.bsi_field_adjoint(torch.from_numpy(g).to(dev()), spacing)
    torch.cuda.synchronize()
    grid = synth.grid_shape(shape, spacing)
    pts = synth.sample_grid_points(grid, 400, seed=4)
    want = oracle.adjoint_points(g, spacing, pts)
    got = d[torch.from_numpy(pts[:, 2]), torch.from_numpy(pts[:, 1]), torch.from_numpy(pts[:, 0])]
    got = got.double().cpu().numpy()
    # scale: the largest |dphi| over the whole grid (GPU) bounds the oracle's
    scale = float(d.abs().max())
    assert np.max(np.abs(got - want)) <= ADJ_TOL * scale


def test_batched_64_instances_sampled():
    geoms = synth.batch_geometries(64, seed=5)
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    total = sum(int(np.prod(s)) for s in shapes)
    assert 1.0e8 < total < 2.5e8
    phis = [synth.uniform_phi(s, d, -3, 3, seed=500 + i) for i, (s, d) in enumerate(geoms)]
    outs = P.bsi_field_forward_batched([torch.from_numpy(p).to(dev()) for p in phis], shapes, spacings)
    torch.cuda.synchronize()
    for i in range(0, 64, 7):
        got, want = _sampled_fwd(phis[i], shapes[i], spacings[i], outs[i], npts=300, seed=i)
        assert np.max(np.abs(got - want)) <= FWD_TOL * np.abs(phis[i]).max(), i
    # adjoint on a subset of volumes, checked at sampled grid points
    sel = list(range(0, 64, 9))
    grads = [synth.normal_field(shapes[i], seed=600 + i) for i in sel]
    dphis = P.bsi_field_adjoint_batched([torch.from_numpy(g).to(dev()) for g in grads],
                                        [spacings[i] for i in sel])
    torch.cuda.synchronize()
    for k, i in enumerate(sel):
        grid = synth.grid_shape(shapes[i], spacings[i])
        pts = synth.sample_grid_points(grid, 60, seed=i)
        want = oracle.adjoint_points(grads[k], spacings[i], pts)
        got = dphis[k][torch.from_numpy(pts[:, 2]), torch.from_numpy(pts[:, 1]),
                       torch.from_numpy(pts[:, 0])].double().cpu().numpy()
        assert np.max(np.abs(got - want)) <= ADJ_TOL * float(dphis[k].abs().max()), i


def _lipschitz(F):
    L = sum(float(np.max(np.abs(np.diff(F.astype(np.float64), axis=ax)))) for ax in range(3) if F.shape[ax] > 1)
    return L + float(np.max(np.abs(F)))


def test_ct_resample_forward_and_backward_sampled():
    """The bench's resampling workload (CT control grid, 8-blob floating image):
    warped values and the voxel gradient G = dW * grad F~ on sampled voxels, and
    dL/dphi against the oracle's transpose of the GPU's own G at sampled grid
    points."""
    shape, spacing = CT
    phi = synth.gaussian_random_phi(shape, spacing, sigma_vox=3.0, smooth_cells=2.0, seed=2)
    F = synth.blob_image(shape, seed=6)
    pt, Ft = torch.from_numpy(phi).to(dev()), torch.from_numpy(F).to(dev())
    W = P.bsi_resample_forward(pt, shape, spacing, Ft)
    dW = torch.randn(shape, device=dev(), generator=torch.Generator(device=dev()).manual_seed(5))
    nbytes = P.bsi_resample_backward_workspace_bytes(shape, spacing)
    ws = torch.empty(nbytes, dtype=torch.uint8, device=dev())
    dphi = P.bsi_resample_backward(pt, shape, spacing, Ft, dW, workspace=ws)
    torch.cuda.synchronize()
    pts = synth.sample_voxels(shape, 3000, seed=6)
    val, grad = oracle.resample_points(phi, shape, spacing, F, pts)
    idx = torch.from_numpy(pts).to(dev())
    got = W[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    tol = 1e-5 * float(np.max(np.abs(phi))) * _lipschitz(F) + 1e-6 * float(np.max(np.abs(F)))
    assert float(np.max(np.abs(got - val))) <= tol
    n = int(np.prod(shape)) * 3
    G = ws[: 4 * n].view(torch.float32).view(shape + (3,))
    gG = G[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    dWs = dW[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    want_G = dWs[:, None] * grad
    # positions within 1e-4 of an integer sit on the interpolant's kinks: left out
    T = oracle.forward_points(phi, shape, spacing, pts)
    frac = (pts + T) - np.floor(pts + T)
    ok = np.all((frac > 1e-4) & (frac < 1 - 1e-4), axis=1)
    assert ok.mean() > 0.9
    assert float(np.max(np.abs(gG - want_G)[ok])) <= 1e-4 * float(np.max(np.abs(want_G))) + 1e-6
    gpts = synth.sample_grid_points(synth.grid_shape(shape, spacing), 300, seed=7)
    want = oracle.adjoint_points(G.cpu().numpy(), spacing, gpts)
    gi = torch.from_numpy(gpts).to(dev())
    gd = dphi[gi[:, 2], gi[:, 1], gi[:, 0]].double().cpu().numpy()
    assert float(np.max(np.abs(gd - want))) <= ADJ_TOL * max(float(np.max(np.abs(want))), 1e-30) * 10


def test_ct_rational_forward_sampled():
    """The bench's non-integer spacing workload: 512x512x300 at 4.7 voxels with
    the lattice shifted by (0.3, 0, 0.9) (z, y, x)."""
    shape, num, den, off = (300, 512, 512), (47, 47, 47), (10, 10, 10), (3, 0, 9)
    grid = P.rational_grid_shape(shape, num, den, off)
    phi = np.random.default_rng(9).uniform(-3, 3, grid + (3,)).astype(np.float32)
    out = P.bsi_field_forward_rational(torch.from_numpy(phi).to(dev()), shape, num, den, off)
    torch.cuda.synchronize()
    pts = synth.sample_voxels(shape, 3000, seed=9)
    want = oracle.forward_rational_points(phi, shape, num, den, off, pts)
    idx = torch.from_numpy(pts).to(dev())
    got = out[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    assert float(np.max(np.abs(got - want))) <= FWD_TOL * float(np.max(np.abs(phi)))


def test_ct_rational_adjoint_sampled():
    """The adjoint of the non-integer spacing workload (512x512x300 at 4.7 voxels,
    shifted lattice) at sampled control points, including the grid's corners."""
    shape, num, den, off = (300, 512, 512), (47, 47, 47), (10, 10, 10), (3, 0, 9)
    G = synth.normal_field(shape, seed=10)
    dphi = P.bsi_field_adjoint_rational(torch.from_numpy(G).to(dev()), num, den, off)
    torch.cuda.synchronize()
    gpts = synth.sample_grid_points(P.rational_grid_shape(shape, num, den, off), 300, seed=10)
    want = oracle.adjoint_rational_points(G, num, den, off, gpts)
    gi = torch.from_numpy(gpts).to(dev())
    gd = dphi[gi[:, 2], gi[:, 1], gi[:, 0]].double().cpu().numpy()
    assert float(np.max(np.abs(gd - want))) <= ADJ_TOL * max(float(np.max(np.abs(want))), 1e-30) * 10


def test_ct_scalar_zoom_sampled():
    """The bench's scalar workload: a 4x zoom of a 128 x 128 x 75 image (plus
    border) to 512 x 512 x 300, FP32 and BF16."""
    shape, spacing = (300, 512, 512), (4, 4, 4)
    img = synth.blob_image(synth.grid_shape(shape, spacing), seed=7)
    t = torch.from_numpy(img).to(dev())
    z = P.bsi_scalar_forward(t, shape, spacing)
    zb = P.bsi_scalar_forward(t, shape, spacing, out_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    pts = synth.sample_voxels(shape, 3000, seed=8)
    phi = np.zeros(img.shape + (3,), np.float64)
    phi[..., 0] = img
    want = oracle.forward_points(phi, shape, spacing, pts)[:, 0]
    idx = torch.from_numpy(pts).to(dev())
    got = z[idx[:, 2], idx[:, 1], idx[:, 0]].double().cpu().numpy()
    assert float(np.max(np.abs(got - want))) <= FWD_TOL * float(np.max(np.abs(img)))
    for zz in range(0, shape[0], 60):
        assert torch.equal(zb[zz], z[zz].to(torch.bfloat16))
