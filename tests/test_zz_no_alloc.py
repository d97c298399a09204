"""The allocation-free solve entry point, called through the C ABI.

dts_solve_noalloc serves callers that cannot allocate device memory and so
cannot pass a workspace (for example code inside a host framework that owns
every device allocation, or a latency-critical loop under a fixed memory
budget): it runs the same solve on a scratch array inside the library.  This
file is collected last so that a failure here never hides the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def _problem(H, W, seed):
    p = workloads.random_problem(H, W, C=3, seed=seed)
    d = _dev()
    return (torch.from_numpy(p.guide).to(d), torch.from_numpy(p.target).to(d), torch.from_numpy(p.conf).to(d),
            float(p.target.max() - p.target.min()))


def _call(lib, g, t, c, prm, out):
    gd = dts.guide_desc(g)
    pc = prm.c()
    return lib.dts_solve_noalloc(ctypes.byref(gd), t.data_ptr(), dts.F32, c.data_ptr(), None, ctypes.byref(pc),
                                 out.data_ptr(), torch.cuda.current_stream().cuda_stream)


def test_noalloc_matches_workspace_solve_on_consecutive_calls():
    lib = dts.load()
    prm = dts.Params(lam=0.99, sigma_s=16.0, sigma_r=0.1, iterations=6)
    problems = [_problem(300, 413, 71), _problem(157, 222, 72)]
    for g, t, c, rng in problems:
        ref = dts.dts_solve(g, t, c, prm)
        for _ in range(2):  # two calls in a row on the shared scratch array
            out = torch.full_like(t, float("nan"))
            assert _call(lib, g, t, c, prm, out) == 0
            torch.cuda.synchronize()
            assert dts.dts_last_status() == 0
            err = float((out - ref).abs().max())
            assert err <= TOL * rng, err


# modes whose working planes differ: conjugate gradients (three more planes and FP64 scalars), the
# support-weighted confidence (its own plane), FP16 distances (and their strip-tiled copy), and a
# column tall enough for the chained vertical pass (its control words and chunk tuples)
CONFIGS = {
    "cg": ((173, 250), dict(update=dts.UPDATE_CG)),
    "support": ((173, 250), dict(conf_mode=dts.CONF_SUPPORT, update=dts.UPDATE_JACOBI)),
    "f16": ((173, 250), dict(dist_dtype=dts.F16)),
    "chain": ((2300, 40), dict()),
}


@pytest.mark.parametrize("name", list(CONFIGS))
def test_noalloc_after_a_call_of_another_mode_and_size(name):
    """Every plane a solve reads is written by that solve first: a mode run right after a call of
    another mode and size on the shared array matches the workspace solve, twice in a row."""
    lib = dts.load()
    other = "chain" if name != "chain" else "cg"
    (H0, W0), kw0 = CONFIGS[other]
    g0, t0, c0, _ = _problem(H0 + 11, W0 + 7, 80)
    p0 = dts.Params(lam=0.99, sigma_s=16.0, sigma_r=0.1, iterations=4, **kw0)
    assert _call(lib, g0, t0, c0, p0, torch.empty_like(t0)) == 0
    (H, W), kw = CONFIGS[name]
    g, t, c, rng = _problem(H, W, 81)
    prm = dts.Params(lam=0.99, sigma_s=16.0, sigma_r=0.1, iterations=5, **kw)
    ref = dts.dts_solve(g, t, c, prm)
    for _ in range(2):
        out = torch.full_like(t, float("nan"))
        assert _call(lib, g, t, c, prm, out) == 0
        torch.cuda.synchronize()
        assert dts.dts_last_status() == 0
        err = float((out - ref).abs().max())
        assert err <= TOL * rng, (name, err)


def test_noalloc_rejects_problems_beyond_its_scratch():
    lib = dts.load()
    cap = lib.dts_noalloc_max_workspace()
    assert cap == 16 << 20
    g, t, c, _ = _problem(1100, 1000, 73)  # 16 B per padded pixel at FP32 distances > 16 MiB
    prm = dts.Params(iterations=2)
    assert dts.workspace_size(g, prm) > cap
    out = torch.empty_like(t)
    assert _call(lib, g, t, c, prm, out) == 3  # DTS_ERR_WORKSPACE
    prm.save_checkpoints = 1
    g2, t2, c2, _ = _problem(64, 64, 74)
    assert _call(lib, g2, t2, c2, prm, torch.empty_like(t2)) == 2  # DTS_ERR_UNSUPPORTED
