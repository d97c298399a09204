"""Failure detection without a GPU fault.  A host-requested, one-shot injection makes one bounded
device-side wait of the hot path run out (about a millisecond under injection): the strip kernel's
wait for a slab load that was left out, the streaming row kernel's wait for a row copy that was left out, the chained vertical pass's wait for a strip composition
that never comes (one chunk does not count its arrival), the resident solve's grid barrier
(one CTA leaves out its arrival), and the persistent batched solve's wait for an image's previous
stage (one job does not count itself done).  Each time the kernel records DTS_ERR_TIMEOUT in the device
status word and still completes; the status reads back once and is then clear, and the next call
on the same workspace matches the oracle again."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu

INJECT_TMA_SKIP, INJECT_CHAIN_SKIP, INJECT_BARRIER_SKIP, INJECT_QUEUE_SKIP, INJECT_STAGE_SKIP = 1, 2, 3, 4, 5
TIMEOUT = 5


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def launched(fn):
    """Runs fn and returns the names of the library kernels it launched."""
    dts.dts_profile(1)
    try:
        fn()
        torch.cuda.synchronize()
        return {r[0] for r in dts.dts_profile_read()}
    finally:
        dts.dts_profile(0)


def check_filter(prob, out, prm):
    ref = oracle.filter(prob.guide, prob.target, prm.sigma_s, prm.sigma_r, passes=prm.passes)
    assert float(np.abs(out.cpu().numpy() - ref).max()) <= 1e-4 * float(np.ptp(prob.target))


# 100 x 200: the strip kernel covers the 25 strips in one round; 3000 x 70: the tall-column
# clusters cover the 3 strips in one round; 12000 x 70: chains of 94 chunks; 20 x 9000: the
# streaming row kernel (CTA 0's first row)
@pytest.mark.parametrize("H,W,kind,kernel", [(100, 200, INJECT_TMA_SKIP, "col_strip_kernel"),
                                             (3000, 70, INJECT_TMA_SKIP, "col_tall_kernel"),
                                             (12000, 70, INJECT_CHAIN_SKIP, "col_chain_kernel"),
                                             (20, 9000, INJECT_STAGE_SKIP, "row_stream_kernel")])
def test_pass_wait_reports_timeout_and_recovers(H, W, kind, kernel):
    d = dev()
    lib = dts.load()
    prob = workloads.random_problem(H, W, C=3, seed=3)
    g = torch.from_numpy(prob.guide).to(d)
    src = torch.from_numpy(prob.target).to(d)
    prm = dts.Params(sigma_s=8.0, sigma_r=0.2, passes=2)
    ws = dts.workspace(g, prm)
    assert dts.dts_last_status() == 0
    assert lib.dts_debug_inject(kind) == 0
    assert kernel in launched(lambda: dts.dts_filter(g, src, prm, ws=ws))
    assert dts.dts_last_status() == TIMEOUT  # then cleared
    assert dts.dts_last_status() == 0
    out = dts.dts_filter(g, src, prm, ws=ws)
    assert dts.dts_last_status() == 0
    check_filter(prob, out, prm)
    assert lib.dts_debug_inject(7) == 1  # unknown kind: DTS_ERR_INVALID_ARG
    assert lib.dts_debug_inject(0) == 0


def test_chained_adjoint_wait_reports_timeout_and_recovers():
    """The chained vertical adjoint (a tuned plan for this height; every pass input kept, so the
    first chained launch after the request is the backward's)."""
    d = dev()
    lib = dts.load()
    H, W = 4520, 40
    dts.autotune_import("bcol %d 16 16 -1\n" % H)
    rng = np.random.default_rng(45)
    I = rng.random((3, H, W)).astype(np.float32)
    t = rng.normal(size=(H, W)).astype(np.float32)
    c = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    gz = rng.normal(size=(H, W)).astype(np.float32)
    prm = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=2, save_checkpoints=2)
    g, tt, cc, gzt = (torch.from_numpy(x).to(d) for x in (I, t, c, gz))
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, tt, cc, prm, ws=ws)
    assert dts.dts_last_status() == 0
    assert lib.dts_debug_inject(INJECT_CHAIN_SKIP) == 0
    assert "col_bwd_chain_kernel" in launched(lambda: dts.dts_solve_backward(g, tt, cc, prm, ws, gzt))
    assert dts.dts_last_status() == TIMEOUT
    assert dts.dts_last_status() == 0
    gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, gzt)
    assert dts.dts_last_status() == 0
    ref = oracle.solve_backward(I, t, c, gz, lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=2)
    for got, name in ((gt, "t"), (gc, "c"), (gg, "guide")):
        assert float(np.abs(got.cpu().numpy() - ref[name]).max()) <= 1e-3 * float(np.abs(ref[name]).max()), name


def test_resident_grid_barrier_reports_timeout_and_recovers(monkeypatch):
    """The resident solve (DTS_RESIDENT=1, 2^20 pixels or more): CTA 0 leaves out its first arrival
    at the grid-wide barrier; every wait there runs out, raises the abort word (no later barrier
    waits) and the kernel ends."""
    d = dev()
    lib = dts.load()
    monkeypatch.setenv("DTS_RESIDENT", "1")
    prob = workloads.random_problem(1024, 1100, C=3, seed=9)
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=3)
    g, t, c = (torch.from_numpy(x).to(d) for x in (prob.guide, prob.target, prob.conf))
    ws = dts.workspace(g, prm)
    assert lib.dts_debug_inject(INJECT_BARRIER_SKIP) == 0
    assert "resident_solve_kernel" in launched(lambda: dts.dts_solve(g, t, c, prm, ws=ws))
    assert dts.dts_last_status() == TIMEOUT
    assert dts.dts_last_status() == 0
    z = dts.dts_solve(g, t, c, prm, ws=ws)
    assert dts.dts_last_status() == 0
    ref = oracle.solve(prob.guide, prob.target, prob.conf, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=3)
    assert float(np.abs(z.cpu().numpy() - ref).max()) <= 1e-4 * float(np.ptp(prob.target))


def test_batched_queue_wait_reports_timeout_and_recovers():
    d = dev()
    lib = dts.load()
    wl = workloads.workload_batched(seed=12, n=4, hmin=20, hmax=120, wmin=20, wmax=160)
    g = [torch.from_numpy(p.guide).to(d) for p in wl.problems]
    t = [torch.from_numpy(p.target).to(d) for p in wl.problems]
    c = [torch.from_numpy(p.conf).to(d) for p in wl.problems]
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=2)
    dts.autotune_import("batch 0\n")
    assert lib.dts_debug_inject(INJECT_QUEUE_SKIP) == 0
    assert "batched_solve_kernel" in launched(lambda: dts.dts_solve_batched(g, t, c, prm))
    assert dts.dts_last_status() == TIMEOUT
    assert dts.dts_last_status() == 0
    outs = dts.dts_solve_batched(g, t, c, prm)
    assert dts.dts_last_status() == 0
    for i, p in enumerate(wl.problems):
        ref = oracle.solve(p.guide, p.target, p.conf, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=2)
        assert float(np.abs(outs[i].cpu().numpy() - ref).max()) <= 1e-4 * float(np.ptp(p.target)), i
