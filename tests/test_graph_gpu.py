"""The batched forward + adjoint captured once in a CUDA graph and replayed:
the library allocates and synchronises nothing inside the calls."""
import numpy as np
import pytest
import torch

import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu


def test_batched_fwd_adj_graph_replay_matches_eager():
    geoms = synth.batch_geometries(16, seed=61, xy_range=(16, 96), z_range=(16, 64))
    shapes = [g[0] for g in geoms]
    spacings = [g[1] for g in geoms]
    phis = [torch.from_numpy(synth.uniform_phi(s, d, -3, 3, seed=700 + i)).to(dev())
            for i, (s, d) in enumerate(geoms)]
    grads = [torch.from_numpy(synth.normal_field(s, seed=800 + i)).to(dev()) for i, s in enumerate(shapes)]
    outs = [torch.empty(s + (3,), device=dev()) for s in shapes]
    dphis = [torch.empty(synth.grid_shape(s, d) + (3,), device=dev()) for s, d in geoms]
    ws = torch.empty(P.bsi_batched_adjoint_workspace_bytes(shapes, spacings), dtype=torch.uint8, device=dev())

    def step():
        P.bsi_field_forward_batched(phis, shapes, spacings, outs=outs)
        P.bsi_field_adjoint_batched(grads, spacings, outs=dphis, workspace=ws)

    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        step()  # warm-up outside capture: per-device launch facts are cached here
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    eager_f = [o.clone() for o in outs]
    eager_d = [d.clone() for d in dphis]
    for o in outs:
        o.zero_()
    for d in dphis:
        d.zero_()

    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        step()
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, eager_f):
        assert torch.equal(a, b)
    for a, b in zip(dphis, eager_d):
        assert torch.equal(a, b)
    # new inputs are picked up by the replay
    for p in phis:
        p.mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(outs, eager_f):
        assert torch.allclose(a, 2 * b, rtol=1e-6, atol=1e-5)
