"""Helpers shared by the GPU tests: run the CUDA path through the binding and
compare with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

from concurrent.futures import ThreadPoolExecutor

import numpy as np
import torch

import oracle
import paper_2004_05962_gb300 as P

# Acceptance tolerances (FP32 path vs FP64 oracle):
#   forward: max|err| <= 1e-5 * max|phi|;  adjoint: max|err| <= 1e-5 * max|oracle dphi|.
FWD_TOL = 1e-5
ADJ_TOL = 1e-5
# BF16 storage: round-to-nearest-even of the FP32 result, |x - rne(x)| <= 2^-8 |x|.
BF16_REL = 2.0 ** -8


def dev():
    return torch.device("cuda", 0)


def gpu_forward(phi_np, shape, spacing, dtype=torch.float32, out=None):
    phi = torch.from_numpy(np.ascontiguousarray(phi_np)).to(dev())
    t = P.bsi_field_forward(phi, shape, spacing, out=out, out_dtype=dtype)
    torch.cuda.synchronize()
    return t


def gpu_adjoint(g_np, spacing):
    g = torch.from_numpy(np.ascontiguousarray(g_np)).to(dev())
    t = P.bsi_field_adjoint(g, spacing)
    torch.cuda.synchronize()
    return t


def fwd_err(got, phi, shape, spacing):
    want = oracle.forward(phi, shape, spacing)
    err = float(np.max(np.abs(got.double() .cpu().numpy() - want))) if want.size else 0.0
    return err, FWD_TOL * float(np.max(np.abs(phi)))


def adj_err(got, g, spacing):
    want = oracle.adjoint(g, spacing)
    err = float(np.max(np.abs(got.double().cpu().numpy() - want)))
    return err, ADJ_TOL * max(float(np.max(np.abs(want))), 1e-30)


# ------------------------------------------------------------------ full-volume checks
#
# The workloads the benchmark times are checked at every voxel / control point.
# The oracle's point-wise forms evaluate Eq. 1 (or its transpose) at a list of
# voxels with the whole control grid, so a volume is walked a chunk of z-planes
# at a time and never needs a full FP64 copy on the host.

def plane_points(Y, X, z0, z1):
    """Every voxel of planes [z0, z1) as (x, y, z) rows, in memory order."""
    z, y, x = np.meshgrid(np.arange(z0, z1), np.arange(Y), np.arange(X), indexing="ij")
    return np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1).astype(np.int64)


def oracle_by_planes(fn, shape, planes=16, threaded=False):
    """Yields (z0, z1, want) over the volume, want = fn(points of planes
    [z0, z1)) reshaped to [z1 - z0, Y, X, -1].  ``threaded`` splits each chunk
    over the host cores for the oracle's single-threaded point-wise forms
    (ctypes releases the GIL during the call)."""
    Z, Y, X = (int(s) for s in shape)
    nt = oracle.threads()
    pool = ThreadPoolExecutor(nt) if threaded else None
    try:
        for z0 in range(0, Z, planes):
            z1 = min(Z, z0 + planes)
            pts = plane_points(Y, X, z0, z1)
            if pool is not None:
                want = np.concatenate(list(pool.map(fn, np.array_split(pts, nt))))
            else:
                want = fn(pts)
            yield z0, z1, want.reshape(z1 - z0, Y, X, -1)
    finally:
        if pool is not None:
            pool.shutdown()


class FieldError:
    """max / mean |got - want| over a whole field, and whether every element
    met |got - want| <= rel * |want| + atol."""

    def __init__(self, atol, rel=0.0):
        self.atol, self.rel = atol, rel
        self.max = 0.0
        self.sum = 0.0
        self.n = 0
        self.violations = 0

    def add(self, got, want):
        d = np.abs(got - want)
        if d.size:
            self.max = max(self.max, float(d.max()))
            self.sum += float(d.sum())
            self.n += d.size
            self.violations += int(np.count_nonzero(d > self.rel * np.abs(want) + self.atol))

    @property
    def mean(self):
        return self.sum / max(self.n, 1)

    @property
    def ok(self):
        return self.violations == 0 and self.n > 0

    def __repr__(self):
        return (f"max {self.max:.3e} mean {self.mean:.3e} over {self.n} elements, "
                f"{self.violations} beyond {self.rel:.3g}|want| + {self.atol:.3e}")


def host_planes(t, z0, z1, shape_tail):
    """Planes [z0, z1) of a device tensor as FP64 numpy, shaped [z1 - z0, *shape_tail]."""
    return t[z0:z1].float().cpu().numpy().astype(np.float64).reshape((z1 - z0,) + tuple(shape_tail))


def full_forward_check(phi, shape, spacing, outs, planes=16):
    """Compares each device field in ``outs`` (name -> (tensor, FieldError))
    with the oracle's Eq. 1 at every voxel."""
    Z, Y, X = shape
    fn = lambda pts: oracle.forward_points(phi, shape, spacing, pts)
    for z0, z1, want in oracle_by_planes(fn, shape, planes):
        for t, err in outs.values():
            err.add(host_planes(t, z0, z1, (Y, X, 3)), want)
    return outs


def full_adjoint_check(grad_np, spacing, got, atol_rel=ADJ_TOL):
    """dL/dphi at every control point against the oracle's transpose of Eq. 1;
    the tolerance is atol_rel times the oracle's largest |dphi|."""
    want = oracle.adjoint(grad_np, spacing)
    err = FieldError(atol_rel * max(float(np.max(np.abs(want))), 1e-30))
    err.add(got.double().cpu().numpy(), want)
    return err
