"""The bounds-checked build (BSI_CHECKED): every kernel access is range-tested
in the kernel itself; on the parity cases no check fires and the results match
the release build bit for bit."""
import pytest
import torch

import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import bsi as B
from paper_2004_05962_gb300 import build as Bd
from paper_2004_05962_gb300 import synth
from gpu_util import dev

pytestmark = pytest.mark.gpu

# 64^3 at 5: BF16 rows in tensor-store blocks (24-tile strips), adjoint units of
# two tile-rows; (10, 17, 252) at (4, 6, 3): FP32 rows in blocks of 3 rows
CASES = [((64, 64, 64), (5, 5, 5)), ((9, 8, 140), (3, 5, 13)), ((6, 7, 179), (2, 3, 2)),
         ((5, 4, 130), (2, 2, 64)), ((1, 1, 1), (1, 1, 1)), ((10, 17, 252), (4, 6, 3))]


def _run(phi, shape, spacing, g):
    out = P.bsi_field_forward(phi, shape, spacing)
    o16 = P.bsi_field_forward(phi, shape, spacing, out_dtype=torch.bfloat16)
    d = P.bsi_field_adjoint(g, spacing)
    return out, o16, d, P.bsi_check_device_status()


def test_checked_build_no_violation_and_same_results():
    Bd.build(checked=True)
    try:
        for shape, spacing in CASES:
            phi = torch.from_numpy(synth.uniform_phi(shape, spacing, -2, 2, seed=9)).to(dev())
            g = torch.from_numpy(synth.normal_field(shape, seed=10)).to(dev())
            B.set_checked(True)
            a = _run(phi, shape, spacing, g)
            B.set_checked(False)
            b = _run(phi, shape, spacing, g)
            assert a[3] == 0, f"checked kernels flagged 0x{a[3]:x} on {shape} {spacing}"
            assert b[3] == 0
            for x, y in zip(a[:3], b[:3]):
                assert torch.equal(x, y)
    finally:
        B.set_checked(False)
