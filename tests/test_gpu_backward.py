"""GPU parity of dts_solve_backward (through the C ABI and the autograd Function)
against the FP64 oracle's reverse mode, itself pinned by finite differences and
an autograd restatement.  Tolerance (FP32 arithmetic, long reversed recurrences):
max |g_gpu - g_oracle| <= 1e-3 * max |g_oracle| for every gradient."""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu

GTOL = 1e-3


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def T(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def guide_noisy(H, W, C, seed):
    rng = np.random.default_rng(seed)
    return rng.random((C, H, W)).astype(np.float32)


def close(gpu, ref, what):
    scale = float(np.abs(ref).max()) or 1.0
    err = float(np.abs(gpu - ref).max())
    assert err <= GTOL * scale, f"{what}: {err:.3e} > {GTOL * scale:.3e}"


def run_case(H, W, C=3, K=4, update=dts.UPDATE_GD, norm=dts.NORM_L1, zinit=False, seed=0, passes=3,
             sigma_s=8.0, sigma_r=0.3, dist=dts.F32, keep=1, eps=0.0):
    rng = np.random.default_rng(seed)
    I = guide_noisy(H, W, C, seed)
    t = rng.normal(size=(H, W)).astype(np.float32)
    c = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    gz = rng.normal(size=(H, W)).astype(np.float32)
    z0 = rng.normal(size=(H, W)).astype(np.float32) if zinit else None
    prm = dts.Params(lam=0.9, sigma_s=sigma_s, sigma_r=sigma_r, iterations=K, passes=passes, update=update,
                     norm=norm, dist_dtype=dist, save_checkpoints=keep, charbonnier_eps=eps)
    g, tt, cc = T(I), T(t), T(c)
    zi = T(z0) if zinit else None
    ws = dts.workspace(g, prm, with_backward=True)
    z = dts.dts_solve(g, tt, cc, prm, z_init=zi, ws=ws)
    gt, gc, gg, gz0 = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz), z_init=zi)
    assert dts.dts_last_status() == 0
    kw = dict(lam=0.9, sigma_s=sigma_s, sigma_r=sigma_r, iterations=K, passes=passes, update=update, norm=norm,
              charbonnier_eps=eps)
    if dist == dts.F16:
        return z, gt, gc, gg, gz0, None
    ref = oracle.solve_backward(I, t, c, gz, z_init=z0, **kw)
    zr = oracle.solve(I, t, c, z_init=z0, **kw)
    np.testing.assert_allclose(z.cpu().numpy(), zr, atol=1e-4 * float(np.ptp(t)))
    close(gt.cpu().numpy(), ref["t"], "grad target")
    close(gc.cpu().numpy(), ref["c"], "grad conf")
    close(gg.cpu().numpy(), ref["guide"], "grad guide")
    if zinit:
        close(gz0.cpu().numpy(), ref["z_init"], "grad z_init")
    return z, gt, gc, gg, gz0, ref


@pytest.mark.parametrize("H,W", [(1, 1), (1, 23), (29, 1), (17, 31), (64, 80), (130, 70), (45, 300), (300, 45)])
def test_backward_shapes(H, W):
    run_case(H, W, seed=H * 31 + W)


@pytest.mark.parametrize("H,W", [(64, 80), (300, 45)])
def test_backward_charbonnier(H, W):
    """The reverse mode of the gradient step with the Charbonnier target loss (§4): eps = 1, the
    step's curvature in the stable range (see the forward tests), and with a starting point away
    from the target."""
    run_case(H, W, K=4, seed=H + W + 5, eps=1.0)
    run_case(H, W, K=3, seed=H + W + 6, eps=1.0, zinit=True)


@pytest.mark.parametrize("eps", [0.3, 0.01])
def test_backward_charbonnier_fixed_point(eps):
    """The reverse mode of the fixed point of Eq. 4 with the Charbonnier loss's weight at the
    current iterate (the weight reaches z_k and t through the residual)."""
    run_case(64, 80, K=4, update=dts.UPDATE_JACOBI, seed=71, eps=eps)
    run_case(300, 45, K=3, update=dts.UPDATE_JACOBI, seed=72, eps=eps, zinit=True)


@pytest.mark.parametrize("update", [dts.UPDATE_GD, dts.UPDATE_JACOBI])
def test_backward_kept_pass_inputs(update):
    """save_checkpoints = 2 (every pass input kept, no recompute) gives the same forward and
    the same gradients, bit for bit, as save_checkpoints = 1 (recompute from the iterates)."""
    a = run_case(90, 130, K=3, update=update, seed=21 + update, keep=2)
    b = run_case(90, 130, K=3, update=update, seed=21 + update, keep=1)
    for x, y in zip(a[:5], b[:5]):
        if x is not None:
            assert torch.equal(x, y)


def test_backward_needs_kept_iterates():
    dev()
    prm = dts.Params(iterations=2)
    g = torch.rand((3, 20, 30), device=dev())
    t = torch.rand((20, 30), device=dev())
    ws = dts.workspace(g, prm, with_backward=True)
    with pytest.raises(RuntimeError):
        dts.dts_solve_backward(g, t, t, prm, ws, t)


# columns over 1536 rows: the two-phase vertical adjoint (chunk totals of 64 rows, their
# composition per strip, the replay); rows over 8192: 16 positions per thread in the row adjoint
@pytest.mark.parametrize("H,W,update", [(4500, 40, dts.UPDATE_GD), (9000, 9, dts.UPDATE_JACOBI),
                                        (5, 9000, dts.UPDATE_GD), (3, 10240, dts.UPDATE_JACOBI)])
def test_backward_tall_and_wide(H, W, update):
    run_case(H, W, K=2, update=update, seed=H + W)


def test_backward_limits():
    # rows over 10240 have no backward plan; the forward still runs
    dev()
    prm = dts.Params(iterations=1, save_checkpoints=1)
    g = torch.zeros((3, 2, 10300), device=dev())
    t = torch.zeros((2, 10300), device=dev())
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, t, t, prm, ws=ws)
    with pytest.raises(RuntimeError):
        dts.dts_solve_backward(g, t, t, prm, ws, t)


@pytest.mark.parametrize("update,norm,zinit", [(dts.UPDATE_JACOBI, dts.NORM_L1, False),
                                               (dts.UPDATE_GD, dts.NORM_L2, False),
                                               (dts.UPDATE_JACOBI, dts.NORM_L2, True),
                                               (dts.UPDATE_GD, dts.NORM_L1, True)])
def test_backward_variants(update, norm, zinit):
    run_case(70, 90, update=update, norm=norm, zinit=zinit, seed=5 + update + 2 * norm)


def test_backward_iterations_and_passes():
    run_case(50, 60, K=0, seed=1)
    run_case(50, 60, K=1, passes=1, seed=2)
    run_case(50, 60, K=7, passes=5, seed=3)


def test_backward_larger_multi_cluster():
    run_case(600, 420, K=3, seed=9, sigma_s=20.0)


def test_autograd_function_matches_oracle():
    H, W = 40, 52
    rng = np.random.default_rng(77)
    I = guide_noisy(H, W, 3, 77)
    t = rng.normal(size=(H, W)).astype(np.float32)
    c = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    gz = rng.normal(size=(H, W)).astype(np.float32)
    prm = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3)
    g = T(I).requires_grad_(True)
    tt = T(t).requires_grad_(True)
    cc = T(c).requires_grad_(True)
    z = dts.solve(g, tt, cc, prm)
    (z * T(gz)).sum().backward()
    ref = oracle.solve_backward(I, t, c, gz, lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3)
    close(tt.grad.cpu().numpy(), ref["t"], "autograd t")
    close(cc.grad.cpu().numpy(), ref["c"], "autograd c")
    close(g.grad.cpu().numpy(), ref["guide"], "autograd guide")


def test_autograd_retain_graph_and_unsupported_modes():
    """A second backward through a retained graph gives the same gradients (the workspace holding
    the checkpoints is a saved tensor); modes without a backward are refused in the forward."""
    H, W = 33, 41
    rng = np.random.default_rng(33)
    I = guide_noisy(H, W, 3, 33)
    t = rng.normal(size=(H, W)).astype(np.float32)
    c = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    prm = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3)
    tt = T(t).requires_grad_(True)
    z = dts.solve(T(I), tt, T(c), prm)
    loss = (z * z).sum()
    loss.backward(retain_graph=True)
    first = tt.grad.clone()
    tt.grad = None
    loss.backward()
    assert torch.equal(first, tt.grad)
    for bad in (dict(update=dts.UPDATE_CG), dict(conf_mode=dts.CONF_SUPPORT), dict(filter_kernel=dts.KERNEL_BOX)):
        q = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3, **bad)
        with pytest.raises(ValueError):
            dts.solve(T(I), T(t).requires_grad_(True), T(c), q)


# the guide gradient four pixels per thread (rows of whole 16-byte units: W = 96) and one per
# thread (W = 98), for FP32, BF16 and FP16 guide storage and both distance norms; 16-bit guides
# against the oracle on the stored (rounded) guide
@pytest.mark.parametrize("W", [96, 98])
@pytest.mark.parametrize("gdtype", ["f32", "bf16", "f16"])
@pytest.mark.parametrize("norm", [dts.NORM_L1, dts.NORM_L2])
def test_backward_guide_gradient_layouts(W, gdtype, norm):
    H = 40
    rng = np.random.default_rng(W + 7 * norm + len(gdtype))
    I = guide_noisy(H, W, 3, W + norm)
    t = rng.normal(size=(H, W)).astype(np.float32)
    c = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    gz = rng.normal(size=(H, W)).astype(np.float32)
    g = T(I, {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[gdtype])
    prm = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3, norm=norm, save_checkpoints=1)
    tt, cc = T(t), T(c)
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, tt, cc, prm, ws=ws)
    dts.dts_profile(1)
    gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz))
    torch.cuda.synchronize()
    names = {r[0] for r in dts.dts_profile_read()}
    dts.dts_profile(0)
    assert dts.dts_last_status() == 0
    assert ("guide_grad_kernel<x4>" in names) == (W % 4 == 0), names
    ref = oracle.solve_backward(g.float().cpu().numpy(), t, c, gz, lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3,
                                passes=3, norm=norm)
    close(gt.cpu().numpy(), ref["t"], "grad target")
    close(gc.cpu().numpy(), ref["c"], "grad conf")
    close(gg.cpu().numpy(), ref["guide"], "grad guide")


def test_backward_fp16_distances_runs_and_agrees_roughly():
    z, gt, gc, gg, _, _ = run_case(64, 96, dist=dts.F16, seed=4)
    _, gt32, gc32, gg32, _, _ = run_case(64, 96, seed=4)
    for a, b in ((gt, gt32), (gc, gc32)):
        a, b = a.cpu().numpy(), b.cpu().numpy()
        assert np.abs(a - b).max() <= 2e-2 * np.abs(b).max()


def test_backward_depth_sr_batch_full_size():
    """The x16 depth super-resolution workload (8 x 2048 x 1536, K = 10) at full size: every
    gradient of every image against the oracle's reverse mode."""
    wl = workloads.make(2)
    q = wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes,
                     save_checkpoints=1)
    rng = np.random.default_rng(2002)
    for i, p in enumerate(wl.problems):
        gz = rng.normal(size=p.target.shape).astype(np.float32)
        g, tt, cc = T(p.guide), T(p.target), T(p.conf)
        ws = dts.workspace(g, prm, with_backward=True)
        dts.dts_solve(g, tt, cc, prm, ws=ws)
        gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz))
        ref = oracle.solve_backward(p.guide, p.target, p.conf, gz, lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r,
                                    iterations=q.iterations, passes=q.passes)
        close(gt.cpu().numpy(), ref["t"], f"image {i} grad target")
        close(gc.cpu().numpy(), ref["c"], f"image {i} grad conf")
        close(gg.cpu().numpy(), ref["guide"], f"image {i} grad guide")
        del ws


def test_backward_depth_sr_reduced_finite_differences():
    """The x16 depth-SR generator at 256 x 192 (K = 10, sigma_s = 320): GPU gradients against
    central finite differences of the FP64 oracle's loss <g, z_K> at 64 random entries of each
    of the target, the confidence and the guide."""
    wl = workloads.workload_depth_sr(batch=1, H=192, W=256)
    p, q = wl.problems[0], wl.params
    kw = dict(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
    prm = dts.Params(save_checkpoints=1, **{("lam" if k == "lam" else k): v for k, v in kw.items()})
    rng = np.random.default_rng(192)
    gz = rng.normal(size=p.target.shape)
    g, tt, cc = T(p.guide), T(p.target), T(p.conf)
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, tt, cc, prm, ws=ws)
    gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz.astype(np.float32)))
    gt, gc, gg = gt.cpu().numpy(), gc.cpu().numpy(), gg.cpu().numpy()
    I0, t0, c0 = (x.astype(np.float64) for x in (p.guide, p.target, p.conf))

    def loss(I, t, c):
        return float(np.sum(gz * oracle.solve(I, t, c, **kw)))

    H, W = t0.shape
    for name, grad, h in (("target", gt, 1e-3), ("conf", gc, 1e-4)):
        for _ in range(64):
            y, x = int(rng.integers(H)), int(rng.integers(W))
            a, b = t0.copy(), c0.copy()
            arr = a if name == "target" else b
            arr[y, x] += h
            lp = loss(I0, a, b)
            arr[y, x] -= 2 * h
            lm = loss(I0, a, b)
            fd = (lp - lm) / (2 * h)
            assert abs(grad[y, x] - fd) <= GTOL * np.abs(grad).max(), (name, y, x, grad[y, x], fd)
    # guide: entries whose neighbour differences (the L1 kinks) are all far from zero
    h = 1e-6
    checked = 0
    while checked < 64:
        k, y, x = int(rng.integers(I0.shape[0])), int(rng.integers(1, H - 1)), int(rng.integers(1, W - 1))
        diffs = [I0[k, y, x] - I0[k, y, x - 1], I0[k, y, x + 1] - I0[k, y, x], I0[k, y, x] - I0[k, y - 1, x],
                 I0[k, y + 1, x] - I0[k, y, x]]
        if min(abs(d) for d in diffs) < 100 * h:
            continue
        Ip = I0.copy()
        Ip[k, y, x] += h
        lp = loss(Ip, t0, c0)
        Ip[k, y, x] -= 2 * h
        lm = loss(Ip, t0, c0)
        fd = (lp - lm) / (2 * h)
        assert abs(gg[k, y, x] - fd) <= GTOL * np.abs(gg).max(), ("guide", k, y, x, gg[k, y, x], fd)
        checked += 1


def test_backward_multispectral_reduced():
    """The 16-band multispectral generator at 1200 x 1200 (K = 10): every gradient against the
    oracle's reverse mode."""
    wl = workloads.make(4, H=1200, W=1200)
    p, q = wl.problems[0], wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes,
                     save_checkpoints=2)
    gz = np.random.default_rng(1200).normal(size=p.target.shape).astype(np.float32)
    g, tt, cc = T(p.guide), T(p.target), T(p.conf)
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, tt, cc, prm, ws=ws)
    gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz))
    assert dts.dts_last_status() == 0
    ref = oracle.solve_backward(p.guide, p.target, p.conf, gz, lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r,
                                iterations=q.iterations, passes=q.passes)
    close(gt.cpu().numpy(), ref["t"], "grad target")
    close(gc.cpu().numpy(), ref["c"], "grad conf")
    close(gg.cpu().numpy(), ref["guide"], "grad guide")


@pytest.mark.parametrize("H,W", [(10000, 64), (64, 10000)])
def test_backward_multispectral_full_size_slices(H, W):
    """The multispectral generator on slices that run the full 10000 x 10000 image's backward
    plans (the 10000-row two-phase vertical adjoint; 10000-column rows), K = 10 with every pass input
    kept, as the bench runs it: every gradient against the oracle's reverse mode."""
    rng = np.random.Generator(np.random.PCG64(1004))
    p = workloads.multispectral_image(H, W, rng, bands=16, gy=max(1, H // 100), gx=max(1, W // 100))
    q = workloads.make(4, H=8, W=8).params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes,
                     save_checkpoints=2)
    gz = np.random.default_rng(H + W).normal(size=p.target.shape).astype(np.float32)
    g, tt, cc = T(p.guide), T(p.target), T(p.conf)
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, tt, cc, prm, ws=ws)
    gt, gc, gg, _ = dts.dts_solve_backward(g, tt, cc, prm, ws, T(gz))
    assert dts.dts_last_status() == 0
    ref = oracle.solve_backward(p.guide, p.target, p.conf, gz, lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r,
                                iterations=q.iterations, passes=q.passes)
    close(gt.cpu().numpy(), ref["t"], "grad target")
    close(gc.cpu().numpy(), ref["c"], "grad conf")
    close(gg.cpu().numpy(), ref["guide"], "grad guide")


# the vertical adjoint's chain shapes (rows per thread, warps per CTA), each through a tuned plan
# ("bcol H items warps -1") for a height no other test uses
@pytest.mark.parametrize("H,items,warps", [(4501, 8, 16), (4502, 8, 8), (4503, 16, 8), (4504, 8, 32),
                                           (4505, 16, 16)])
def test_backward_chain_shapes(H, items, warps):
    dts.autotune_import("bcol %d %d %d -1\n" % (H, items, warps))
    assert ("bcol %d %d %d -1" % (H, items, warps)) in dts.autotune_export()
    run_case(H, 40, K=2, update=dts.UPDATE_GD, seed=H, keep=2)


# the two-phase vertical adjoint (chunk totals, strip composition, replay: "bcol H items warps
# -5"): every shape on a column of several chunks and a ragged last chunk, one chunk alone, FP16
# distances, and W not a multiple of the 32-column strip
@pytest.mark.parametrize("H,W,items,warps,dist", [(4511, 40, 8, 16, dts.F32), (4512, 40, 16, 8, dts.F32),
                                                  (4513, 40, 8, 8, dts.F32), (4514, 40, 16, 16, dts.F32),
                                                  (4515, 40, 8, 32, dts.F32), (100, 33, 8, 16, dts.F32),
                                                  (1999, 70, 8, 16, dts.F16)])
def test_backward_split_shapes(H, W, items, warps, dist):
    dts.autotune_import("bcol %d %d %d -5\n" % (H, items, warps))
    assert ("bcol %d %d %d -5" % (H, items, warps)) in dts.autotune_export()
    if dist == dts.F16:
        # FP16 distances: the split adjoint against the one-cluster adjoint on the same planes
        dts.dts_profile(1)
        z, gt, gc, gg, _, _ = run_case(H, W, K=2, update=dts.UPDATE_JACOBI, seed=H, keep=2, dist=dist)
        names = {r[0] for r in dts.dts_profile_read()}
        dts.dts_profile(0)
        assert {"col_bwd_agg_kernel", "col_bwd_apply_kernel"} <= names
        dts.autotune_import("bcol %d 16 16 8\n" % H)
        z2, gt2, gc2, gg2, _, _ = run_case(H, W, K=2, update=dts.UPDATE_JACOBI, seed=H, keep=2, dist=dist)
        assert torch.equal(z, z2)
        for a_, b_ in ((gt, gt2), (gc, gc2), (gg, gg2)):
            scale = float(b_.abs().max()) + 1e-30
            assert float((a_ - b_).abs().max()) <= 1e-4 * scale
        return
    dts.dts_profile(1)
    run_case(H, W, K=2, update=dts.UPDATE_GD, seed=H, keep=2)
    names = {r[0] for r in dts.dts_profile_read()}
    dts.dts_profile(0)
    assert {"col_bwd_agg_kernel", "col_bwd_apply_kernel"} <= names


def test_backward_into_caller_tensors():
    """dts_solve_backward writing into the caller's gradient tensors gives the same bits as into
    tensors it allocates (what a pipelined caller reuses step after step); the guide gradient
    can be left out."""
    rng = np.random.default_rng(61)
    H, W = 97, 130
    g = T(guide_noisy(H, W, 3, 61))
    t, c = T(rng.random((H, W))), T(rng.uniform(0.1, 1.0, (H, W)))
    gz = T(rng.standard_normal((H, W)))
    prm = dts.Params(lam=0.9, sigma_s=8.0, sigma_r=0.3, iterations=3, save_checkpoints=2)
    ws = dts.workspace(g, prm, with_backward=True)
    dts.dts_solve(g, t, c, prm, ws=ws)
    gt, gc, gg, _ = dts.dts_solve_backward(g, t, c, prm, ws, gz)
    outs = (torch.full_like(t, 7.0), torch.full_like(t, 7.0), torch.full_like(g, 7.0), None)
    r = dts.dts_solve_backward(g, t, c, prm, ws, gz, outs=outs)
    assert dts.dts_last_status() == 0
    assert r[0] is outs[0] and r[1] is outs[1] and r[2] is outs[2]
    assert torch.equal(outs[0], gt) and torch.equal(outs[1], gc) and torch.equal(outs[2], gg)
    o2 = (torch.full_like(t, 7.0), torch.full_like(t, 7.0), None, None)
    dts.dts_solve_backward(g, t, c, prm, ws, gz, outs=o2)
    assert torch.equal(o2[0], gt) and torch.equal(o2[1], gc)
