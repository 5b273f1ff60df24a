"""Failure detection without a GPU fault: a bulk copy that never arrives makes
the kernels' bounded mbarrier wait run out; the warp records the timeout bit in
the device status word and returns, and the context stays usable."""
import time

import numpy as np
import pytest
import torch

import oracle
import paper_2004_05962_gb300 as P
from paper_2004_05962_gb300 import bsi as B
from paper_2004_05962_gb300 import synth
from gpu_util import FWD_TOL, dev

pytestmark = pytest.mark.gpu


def test_lost_copy_is_reported_and_the_context_survives():
    torch.cuda.init()
    assert P.bsi_check_device_status() == 0          # clean start (reads and clears)
    t0 = time.time()
    P.bsi_selftest_lost_copy()
    flags = P.bsi_check_device_status()              # synchronises
    waited = time.time() - t0
    assert flags & B.DEVICE_FLAG_TIMEOUT, flags
    assert waited < 30.0, waited                      # bounded: ~2 s at most by construction
    assert P.bsi_check_device_status() == 0          # the word was cleared by the read
    # the context still computes correctly
    shape, spacing = (20, 24, 40), (4, 3, 5)
    phi = synth.uniform_phi(shape, spacing, -2, 2, seed=91)
    got = P.bsi_field_forward(torch.from_numpy(phi).to(dev()), shape, spacing)
    torch.cuda.synchronize()
    err = float(np.max(np.abs(got.double().cpu().numpy() - oracle.forward(phi, shape, spacing))))
    assert err <= FWD_TOL * float(np.max(np.abs(phi)))
    assert P.bsi_check_device_status() == 0
