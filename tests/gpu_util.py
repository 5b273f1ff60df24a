"""Helpers shared by the GPU tests: run the CUDA path through the binding and
compare with the FP64 oracle on the same seeded inputs."""
from __future__ import annotations

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
