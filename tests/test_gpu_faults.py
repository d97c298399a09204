"""Failure detection without a GPU fault: a host-requested injection makes one CTA's
TMA tile never arrive; its bounded wait gives up after about a millisecond, the
kernel records DTS_ERR_TIMEOUT in the device status word and still completes,
and the library keeps working afterwards."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_recovers():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = torch.device("cuda:0")
    lib = dts.load()
    prob = workloads.random_problem(100, 200, C=3, seed=3)
    g = torch.from_numpy(prob.guide).to(d)
    src = torch.from_numpy(prob.target).to(d)
    prm = dts.Params(sigma_s=8.0, sigma_r=0.2, passes=1)
    assert dts.dts_last_status() == 0
    assert lib.dts_debug_inject(1) == 0
    dts.dts_filter(g, src, prm)
    assert dts.dts_last_status() == 5  # DTS_ERR_TIMEOUT, then cleared
    assert dts.dts_last_status() == 0
    out = dts.dts_filter(g, src, prm)
    assert dts.dts_last_status() == 0
    ref = oracle.filter(prob.guide, prob.target, 8.0, 0.2, passes=1)
    assert float(np.abs(out.cpu().numpy() - ref).max()) <= 1e-4 * float(np.ptp(prob.target))
    assert lib.dts_debug_inject(7) == 1
