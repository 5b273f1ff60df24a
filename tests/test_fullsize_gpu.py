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
