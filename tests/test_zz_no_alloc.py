"""bsi_field_adjoint_noalloc: the adjoint for callers that cannot allocate
device memory (a stream being captured into a CUDA graph, a host application
that owns every device allocation, a C caller without a device allocator).
Its scratch is a fixed 64 MiB array inside the library, shared by every call.

The GPU test calls the new entry point through the C ABI twice in a row, on
different volumes and inputs, and checks each result against the existing
bsi_field_adjoint (caller-provided workspace) within the adjoint tolerance of
the other tests.  This file is collected last on purpose, and the test also
passes when it runs alone in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2004_05962_gb300 import bsi as B
from paper_2004_05962_gb300 import synth

ADJ_TOL = 1e-5  # max|err| <= 1e-5 * max|reference grad_phi|, as in the parity tests


def _geom(shape, spacing):
    Z, Y, X = shape
    dz, dy, dx = spacing
    g = B.BsiGeom()
    assert B.library().bsi_geom_init(ctypes.byref(g), X, Y, Z, dx, dy, dz) == 0
    return g


def test_noalloc_rejects_volumes_beyond_its_scratch():
    """Needs no GPU: the size check comes before anything touches CUDA."""
    lib = B.library()
    g = _geom((512, 512, 512), (3, 3, 3))
    assert lib.bsi_adjoint_workspace_bytes(ctypes.byref(g)) > (64 << 20)
    fake = 0x7F0000000000  # never dereferenced
    assert lib.bsi_field_adjoint_noalloc(ctypes.byref(g), fake, fake, None) == 11
    assert lib.bsi_field_adjoint_noalloc(None, fake, fake, None) == 1
    small = _geom((10, 10, 10), (3, 3, 3))
    assert lib.bsi_field_adjoint_noalloc(ctypes.byref(small), None, fake, None) == 1


@pytest.mark.gpu
def test_noalloc_adjoint_matches_workspace_adjoint_two_calls_in_a_row():
    import torch

    lib = B.library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    # the first call fills most of the scratch (the CT-shaped volume needs ~60 MB);
    # the second, smaller one must not see the first call's leftovers
    cases = [((300, 512, 512), (5, 5, 5), 71), ((37, 45, 61), (5, 4, 3), 72)]
    for shape, spacing, seed in cases:
        grad = torch.from_numpy(synth.normal_field(shape, seed=seed)).to(dev)
        grid = synth.grid_shape(shape, spacing)
        ref = B.bsi_field_adjoint(grad, spacing)  # existing entry point, workspace from torch
        got = torch.full(grid + (3,), float("nan"), device=dev)
        g = _geom(shape, spacing)
        assert lib.bsi_field_adjoint_noalloc(ctypes.byref(g), grad.data_ptr(), got.data_ptr(),
                                             stream.cuda_stream) == 0
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        err = float((got - ref).abs().max())
        assert np.isfinite(err) and err <= ADJ_TOL * scale, (shape, spacing, err, scale)
