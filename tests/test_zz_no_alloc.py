"""bsi_field_adjoint_noalloc: the adjoint for callers that cannot allocate
device memory (a stream being captured into a CUDA graph, a host application
that owns every device allocation, a C caller without a device allocator).
Its scratch is a fixed 64 MiB array inside the library, shared by every call.

The GPU tests call the new entry point through the C ABI twice in a row, on
different volumes and inputs, and check each result against the existing
bsi_field_adjoint (caller-provided workspace) within the adjoint tolerance of
the other tests, the smaller one also against the FP64 oracle; they check that
a call leaves the device's free memory unchanged, and that the call captured
in a CUDA graph (after one call outside capture) replays correctly on new
inputs.  This file is collected last on purpose, and its tests also pass when
they run alone in a fresh process.
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


def _noalloc(lib, shape, spacing, grad, out, stream):
    g = _geom(shape, spacing)
    return lib.bsi_field_adjoint_noalloc(ctypes.byref(g), grad.data_ptr(), out.data_ptr(), stream.cuda_stream)


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

    import oracle

    lib = B.library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    # the first call fills most of the scratch (the CT-shaped volume needs ~60 MB);
    # the second, smaller one must not see the first call's leftovers
    cases = [((300, 512, 512), (5, 5, 5), 71), ((37, 45, 61), (5, 4, 3), 72)]
    for k, (shape, spacing, seed) in enumerate(cases):
        g_np = synth.normal_field(shape, seed=seed)
        grad = torch.from_numpy(g_np).to(dev)
        grid = synth.grid_shape(shape, spacing)
        ref = B.bsi_field_adjoint(grad, spacing)  # existing entry point, workspace from torch
        got = torch.full(grid + (3,), float("nan"), device=dev)
        assert _noalloc(lib, shape, spacing, grad, got, stream) == 0
        torch.cuda.synchronize()
        scale = float(ref.abs().max())
        err = float((got - ref).abs().max())
        assert np.isfinite(err) and err <= ADJ_TOL * scale, (shape, spacing, err, scale)
        if k == 1:
            want = oracle.adjoint(g_np, spacing)
            err = float(np.abs(got.double().cpu().numpy() - want).max())
            assert err <= ADJ_TOL * float(np.abs(want).max()), (shape, spacing, err)


@pytest.mark.gpu
def test_noalloc_call_leaves_device_memory_unchanged():
    """After one call (which may load the library's module, and the array with
    it, on this device), a further call changes the device's free memory by
    nothing."""
    import torch

    lib = B.library()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    shape, spacing = (120, 200, 176), (6, 5, 4)
    grad = torch.from_numpy(synth.normal_field(shape, seed=73)).to(dev)
    out = torch.empty(synth.grid_shape(shape, spacing) + (3,), device=dev)
    assert _noalloc(lib, shape, spacing, grad, out, stream) == 0
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info(dev)[0]
    assert _noalloc(lib, shape, spacing, grad, out, stream) == 0
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info(dev)[0] == free0
    ref = B.bsi_field_adjoint(grad, spacing)
    torch.cuda.synchronize()
    assert float((out - ref).abs().max()) <= ADJ_TOL * float(ref.abs().max())


@pytest.mark.gpu
def test_noalloc_captured_in_a_graph_replays_on_new_inputs():
    """One call outside capture, then the call captured into a CUDA graph; two
    replays with different gradients in the captured buffer, each compared with
    bsi_field_adjoint."""
    import torch

    lib = B.library()
    dev = torch.device("cuda", 0)
    shape, spacing = (96, 130, 112), (4, 5, 6)
    grad = torch.from_numpy(synth.normal_field(shape, seed=74)).to(dev)
    out = torch.empty(synth.grid_shape(shape, spacing) + (3,), device=dev)
    assert _noalloc(lib, shape, spacing, grad, out, torch.cuda.current_stream(dev)) == 0
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        assert _noalloc(lib, shape, spacing, grad, out, torch.cuda.current_stream(dev)) == 0
    for seed in (75, 76):
        grad.copy_(torch.from_numpy(synth.normal_field(shape, seed=seed)))
        out.fill_(float("nan"))
        graph.replay()
        ref = B.bsi_field_adjoint(grad, spacing)
        torch.cuda.synchronize()
        err = float((out - ref).abs().max())
        assert np.isfinite(err) and err <= ADJ_TOL * float(ref.abs().max()), (seed, err)
