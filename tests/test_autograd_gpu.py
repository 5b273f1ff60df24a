"""Differentiable BSI: autograd gradients through the hand-written adjoint vs
FP64 finite differences (oracle forward + an FP64 CPU warp)."""
import numpy as np
import pytest
import torch
import torch.nn.functional as F

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import dev, full_adjoint_check

pytestmark = pytest.mark.gpu


def warp(img, u):
    """Trilinear resampling of img [Z, Y, X] at voxel p + u(p), u [Z, Y, X, 3] in
    voxels (channel order x, y, z); zero outside (test harness, not the library)."""
    Z, Y, X = img.shape
    z, y, x = torch.meshgrid(torch.arange(Z, dtype=u.dtype, device=u.device),
                             torch.arange(Y, dtype=u.dtype, device=u.device),
                             torch.arange(X, dtype=u.dtype, device=u.device), indexing="ij")
    gx = 2 * (x + u[..., 0]) / (X - 1) - 1
    gy = 2 * (y + u[..., 1]) / (Y - 1) - 1
    gz = 2 * (z + u[..., 2]) / (Z - 1) - 1
    grid = torch.stack([gx, gy, gz], dim=-1)[None]
    return F.grid_sample(img[None, None], grid, mode="bilinear", padding_mode="zeros",
                         align_corners=True)[0, 0]


def loss_terms(u, W, img, target):
    return (W * u).sum() + ((warp(img, u) - target) ** 2).sum()


def test_linear_loss_gradient_is_adjoint():
    """loss = sum(W * u): d loss / d phi = adjoint(W) exactly (192x192x160, spacing 5)."""
    shape, spacing = (160, 192, 192), (5, 5, 5)
    phi = torch.from_numpy(synth.uniform_phi(shape, spacing, -2, 2, seed=4)).to(dev()).requires_grad_()
    W = torch.from_numpy(synth.normal_field(shape, seed=4)).to(dev())
    u = P.field(phi, shape, spacing)
    (W * u).sum().backward()
    want = P.bsi_field_adjoint(W.contiguous(), spacing)
    torch.cuda.synchronize()
    assert torch.equal(phi.grad, want)


def _config4_inputs():
    """192x192x160 at spacing 5: phi ~ U[-2, 2], W ~ N(0, 1), an 8-blob image and
    a target warped by a second smooth grid (the oracle's field of it)."""
    shape, spacing = (160, 192, 192), (5, 5, 5)
    phi_np = synth.uniform_phi(shape, spacing, -2, 2, seed=4)
    W_np = synth.normal_field(shape, seed=4)
    img_np = synth.blob_image(shape, seed=4)
    phi_star = synth.uniform_phi(shape, spacing, -1.5, 1.5, seed=47)
    tgt = warp(torch.from_numpy(img_np), torch.from_numpy(oracle.forward(phi_star, shape, spacing)).float())
    return shape, spacing, phi_np, W_np, img_np, tgt


def test_config4_linear_loss_gradient_vs_oracle_transpose():
    """loss = sum(W * u) at 192x192x160, spacing 5: d loss / d phi is the
    transpose of Eq. 1 applied to W; the autograd gradient is compared with the
    oracle's transpose at every control point."""
    shape, spacing, phi_np, W_np, _, _ = _config4_inputs()
    phi = torch.from_numpy(phi_np).to(dev()).requires_grad_()
    (torch.from_numpy(W_np).to(dev()) * P.field(phi, shape, spacing)).sum().backward()
    torch.cuda.synchronize()
    err = full_adjoint_check(W_np, spacing, phi.grad)
    assert err.ok, err


def test_config4_full_loss_gradient_vs_oracle_transpose():
    """loss = sum(W * u) + SSD(warp(img, u), target) at 192x192x160, spacing 5:
    dL/du (W plus the warp's gradient, from the harness's grid_sample) is captured
    on its way into the adjoint, and the autograd gradient of phi is compared with
    the oracle's transpose of it at every control point."""
    shape, spacing, phi_np, W_np, img_np, tgt = _config4_inputs()
    phi = torch.from_numpy(phi_np).to(dev()).requires_grad_()
    u = P.field(phi, shape, spacing)
    seen = {}
    u.register_hook(lambda g: seen.setdefault("dLdu", g.detach().clone()))
    L = loss_terms(u, torch.from_numpy(W_np).to(dev()), torch.from_numpy(img_np).to(dev()), tgt.to(dev()))
    L.backward()
    torch.cuda.synchronize()
    dLdu = seen["dLdu"].cpu().numpy()
    assert float(np.abs(dLdu - W_np).max()) > 1e-3   # the SSD term contributes
    err = full_adjoint_check(dLdu, spacing, phi.grad)
    assert err.ok, err


def test_autograd_fd_fp64_32cubed():
    """loss = sum(W*u) + SSD(warp(img, u), target), 32^3 volume, spacing 4: the GPU
    autograd gradient vs central differences of the same loss in FP64 on the CPU."""
    shape, spacing = (32, 32, 32), (4, 4, 4)
    phi_np = synth.uniform_phi(shape, spacing, -2, 2, seed=4)
    W_np = synth.normal_field(shape, seed=44)
    img_np = synth.blob_image(shape, seed=4, nblobs=8, sigma_range=(3.0, 6.0))
    phi_star = synth.uniform_phi(shape, spacing, -1.5, 1.5, seed=45)
    tgt64 = warp(torch.from_numpy(img_np).double(),
                 torch.from_numpy(oracle.forward(phi_star, shape, spacing)))

    phi = torch.from_numpy(phi_np).to(dev()).requires_grad_()
    u = P.field(phi, shape, spacing)
    L = loss_terms(u, torch.from_numpy(W_np).to(dev()), torch.from_numpy(img_np).to(dev()),
                   tgt64.float().to(dev()))
    L.backward()
    grad = phi.grad.double().cpu().numpy()

    W64 = torch.from_numpy(W_np).double()
    img64 = torch.from_numpy(img_np).double()

    def L64(p):
        u64 = torch.from_numpy(oracle.forward(p, shape, spacing))
        return float(loss_terms(u64, W64, img64, tgt64))

    rng = np.random.default_rng(46)
    base = phi_np.astype(np.float64)
    eps = 1e-6  # FP64: small enough that no sample crosses a trilinear kink in practice
    worst = 0.0
    for _ in range(24):
        idx = tuple(int(rng.integers(2, s - 2)) if k < 3 else int(rng.integers(0, 3))
                    for k, s in enumerate(base.shape))
        p1, p2 = base.copy(), base.copy()
        p1[idx] += eps
        p2[idx] -= eps
        fd = (L64(p1) - L64(p2)) / (2 * eps)
        worst = max(worst, abs(fd - grad[idx]))
    assert worst <= 1e-4 * np.abs(grad).max(), (worst, np.abs(grad).max())
