"""GPU parity of the forward path (through the C ABI) against the FP64 oracle.

Tolerance (FP32 arithmetic on the GPU, FP64 in the oracle): the solve and the
filter must agree to max |gpu - oracle| <= 1e-4 * (max t - min t), the bound
stated for this solver; distances to 2e-6 relative (FP32 rounding of a sum
of C absolute differences).  Reduced-precision storage is checked against the
oracle run on the same rounded inputs, with the same bound.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-4

NP_DT = {torch.float32: np.float32, torch.float16: np.float16}


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def rounded(t):
    return t.float().cpu().numpy().astype(np.float64)


def oracle_solve(prob_guide, t, c, prm, **kw):
    return oracle.solve(prob_guide, t, c, lam=prm.lam, sigma_s=prm.sigma_s, sigma_r=prm.sigma_r, step=prm.step,
                        iterations=prm.iterations, passes=prm.passes, norm=prm.norm, update=prm.update,
                        conf_mode=prm.conf_mode, **kw)


def assert_close(z, ref, t, what=""):
    rng = float(np.max(t) - np.min(t)) or 1.0
    err = float(np.abs(z - ref).max()) if z.size else 0.0
    assert err <= TOL * rng, f"{what}: max|gpu-oracle| = {err:.3e} > {TOL * rng:.3e}"


# ---------------------------------------------------------------- distances
# W = 53: one column per thread; W = 52 (rows on 4-element boundaries): four columns per thread
@pytest.mark.parametrize("W", [53, 52])
@pytest.mark.parametrize("gdt", [torch.float32, torch.bfloat16, torch.float16])
@pytest.mark.parametrize("norm", [dts.NORM_L1, dts.NORM_L2])
def test_distances(gdt, norm, W):
    prob = workloads.random_problem(37, W, C=4, seed=2)
    g = to_dev(prob.guide, gdt)
    prm = dts.Params(sigma_s=8.0, sigma_r=0.2, norm=norm)
    dX, dY = dts.dts_domain_transform(g, prm)
    rX, rY = oracle.distances(rounded(g), 8.0, 0.2, norm)
    np.testing.assert_allclose(dX.cpu().numpy(), rX, rtol=2e-6, atol=0)
    np.testing.assert_allclose(dY.cpu().numpy(), rY, rtol=2e-6, atol=0)
    prm.dist_dtype = dts.F16
    hX, hY = dts.dts_domain_transform(g, prm)
    np.testing.assert_allclose(hX.float().cpu().numpy(), rX, rtol=2 ** -10, atol=0)
    np.testing.assert_allclose(hY.float().cpu().numpy(), rY, rtol=2 ** -10, atol=0)


@pytest.mark.parametrize("W", [30, 32])
def test_distances_strided_guide(W):
    prob = workloads.random_problem(20, W, C=3, seed=4)
    big = torch.zeros((3, 25, 40), device=dev())
    big[:, :20, :W] = to_dev(prob.guide)
    view = big[:, :20, :W]
    dX, dY = dts.dts_domain_transform(view, dts.Params())
    rX, rY = oracle.distances(prob.guide, 8.0, 0.2)
    np.testing.assert_allclose(dX.cpu().numpy(), rX, rtol=2e-6)
    np.testing.assert_allclose(dY.cpu().numpy(), rY, rtol=2e-6)


# ---------------------------------------------------------------- filter
# vertical passes: strip CTAs (one per 8 columns, the warp count following the height) up to 2176
# rows -- edges at 1152 / 1153 (segment length 9 -> 17), 1080 (30 warps), 2176 (32 warps) -- and
# clusters above (2177, 4100).  The strip kernel loads and stores through tensor maps; an output
# whose row pitch is not a multiple of 16 bytes (W = 77, 13, ...) takes its plain-load twin for
# the last pass, W = 24 / 12 store through a tensor map into the caller's buffer.
FILTER_SHAPES = [(1, 1), (1, 17), (19, 1), (7, 13), (33, 257), (300, 517), (257, 64), (1000, 77), (1152, 24),
                 (1153, 13), (1080, 31), (2176, 12), (2177, 5), (2100, 40), (3, 9000), (4100, 9), (64, 8193)]


@pytest.mark.parametrize("H,W", FILTER_SHAPES)
def test_filter(H, W):
    prob = workloads.random_problem(H, W, C=3, seed=H * 7 + W)
    prm = dts.Params(sigma_s=12.0, sigma_r=0.3, passes=3)
    g = to_dev(prob.guide)
    src = to_dev(prob.target)
    out = dts.dts_filter(g, src, prm)
    ref = oracle.filter(prob.guide, prob.target, 12.0, 0.3, passes=3)
    assert_close(out.cpu().numpy(), ref, prob.target, f"filter {H}x{W}")


def test_filter_preserves_constants_and_aliases():
    prob = workloads.random_problem(120, 333, C=3, seed=8)
    g = to_dev(prob.guide)
    x = torch.full((120, 333), 0.75, device=dev())
    dts.dts_filter(g, x, dts.Params(), out=x)
    assert float((x - 0.75).abs().max()) <= 1e-6


# ---------------------------------------------------------------- solve
def test_solve_plain_workload():
    wl = workloads.make(0)
    p = wl.problems[0]
    prm = dts.Params(lam=wl.params.lam, sigma_s=wl.params.sigma_s, sigma_r=wl.params.sigma_r,
                     iterations=wl.params.iterations, passes=wl.params.passes)
    z = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm)
    ref = oracle_solve(p.guide, p.target, p.conf, prm)
    assert_close(z.cpu().numpy(), ref, p.target, "plain 256x256")


# (3, 9000) and (2, 16384): rows longer than 8192 apply the update in a horizontal pass with 32
# positions per thread
@pytest.mark.parametrize("H,W", [(1, 1), (1, 40), (40, 1), (31, 45), (129, 300), (700, 263), (1100, 90), (3, 9000),
                                 (2, 16384)])
@pytest.mark.parametrize("update", [dts.UPDATE_GD, dts.UPDATE_JACOBI])
def test_solve_shapes(H, W, update):
    prob = workloads.random_problem(H, W, C=3, seed=H + 3 * W + update)
    prm = dts.Params(lam=0.99, sigma_s=16.0, sigma_r=0.1, iterations=5, update=update)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm)
    assert_close(z.cpu().numpy(), ref, prob.target, f"solve {H}x{W} update={update}")


@pytest.mark.parametrize("variant", ["l2", "support", "zinit", "k0", "checkpoints", "passes1", "passes5"])
def test_solve_variants(variant):
    prob = workloads.random_problem(150, 211, C=3, seed=11)
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=6)
    kw = {}
    z_init = None
    if variant == "l2":
        prm.norm = dts.NORM_L2
    elif variant == "support":
        prm.conf_mode = dts.CONF_SUPPORT
    elif variant == "zinit":
        z_init = np.random.default_rng(3).random(prob.target.shape).astype(np.float32)
        kw["z_init"] = z_init.astype(np.float64)
    elif variant == "k0":
        prm.iterations = 0
    elif variant == "checkpoints":
        prm.save_checkpoints = 1
    elif variant == "passes1":
        prm.passes = 1
    elif variant == "passes5":
        prm.passes = 5
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm,
                      z_init=None if z_init is None else to_dev(z_init))
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm, **kw)
    assert_close(z.cpu().numpy(), ref, prob.target, variant)


@pytest.mark.parametrize("sdt", [torch.bfloat16, torch.float16])
def test_solve_reduced_precision_storage(sdt):
    """Guide and target stored in 16 bits, FP32 arithmetic: against the oracle on
    the same rounded inputs the FP32 bound still holds."""
    prob = workloads.random_problem(200, 300, C=3, seed=12)
    g = to_dev(prob.guide, sdt)
    t = to_dev(prob.target, sdt)
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=8)
    z = dts.dts_solve(g, t, to_dev(prob.conf), prm)
    ref = oracle_solve(rounded(g), rounded(t), prob.conf, prm)
    assert_close(z.cpu().numpy(), ref, rounded(t), f"storage {sdt}")


def test_solve_fp16_distances():
    """FP16 distance planes: checked against the oracle solving on its own FP64
    distances rounded to FP16."""
    prob = workloads.random_problem(180, 260, C=3, seed=13)
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=8, dist_dtype=dts.F16)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    dX, dY = oracle.distances(prob.guide, 8.0, 0.2)
    dX = dX.astype(np.float16).astype(np.float64)
    dY = dY.astype(np.float16).astype(np.float64)
    ref = oracle.solve_d(dX, dY, prob.target, prob.conf, lam=1.0, sigma_s=8.0, iterations=8)
    assert_close(z.cpu().numpy(), ref, prob.target, "fp16 distances")


@pytest.mark.parametrize("H,W", [(180, 260), (1500, 72)])
def test_filter_fp16_distances(H, W):
    """FP16 distance planes in the filter (segments of 9 and of 17 rows in the strip kernel):
    against the oracle filtering with its own FP64 distances rounded to FP16."""
    prob = workloads.random_problem(H, W, C=3, seed=H + W)
    prm = dts.Params(sigma_s=12.0, sigma_r=0.3, passes=3, dist_dtype=dts.F16)
    out = dts.dts_filter(to_dev(prob.guide), to_dev(prob.target), prm)
    dX, dY = oracle.distances(prob.guide, 12.0, 0.3)
    dX = dX.astype(np.float16).astype(np.float64)
    dY = dY.astype(np.float16).astype(np.float64)
    _, a = oracle.schedule(12.0, 3)
    ref = oracle.filter_d(dX, dY, a, prob.target)
    assert_close(out.cpu().numpy(), ref, prob.target, f"fp16 distances {H}x{W}")


def test_solve_full_stereo_workload():
    """The 2880 x 1988, 20-iteration stereo-shaped solve at full size, all outputs."""
    wl = workloads.make(1)
    p = wl.problems[0]
    q = wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
    z = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(p.guide, p.target, p.conf, prm)
    assert_close(z.cpu().numpy(), ref, p.target, "stereo 2880x1988")


# ---------------------------------------------------------------- Charbonnier target loss (§4)
# The gradient step's curvature on the target term is c rho''(r) <= c / eps.  eps = 1 keeps it
# below c (the stable range of the quadratic solve); the paper's eps = 0.001 with confidences
# below 1e-3 keeps eta c / eps < 1.  Outside that range the step overshoots where |z - t| < eps
# and amplifies rounding by up to eta c / eps per iteration, so no elementwise bound holds there.
@pytest.mark.parametrize("H,W", [(37, 53), (300, 257), (1100, 96)])
@pytest.mark.parametrize("eps,cscale", [(1.0, 1.0), (1e-3, 1e-3)])
def test_solve_charbonnier(H, W, eps, cscale):
    prob = workloads.random_problem(H, W, C=3, seed=H + 7 * W)
    c = (prob.conf * cscale).astype(np.float32)
    prm = dts.Params(lam=0.99, sigma_s=8.0, sigma_r=0.2, iterations=10, charbonnier_eps=eps)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(c), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(prob.guide, prob.target, c, prm, charbonnier_eps=eps)
    assert_close(z.cpu().numpy(), ref, prob.target, f"charbonnier eps={eps} {H}x{W}")


def test_solve_charbonnier_box_kernel_and_full_stereo_workload():
    """The Charbonnier step with the box kernel, and on the full 2880 x 1988 stereo workload
    (disparities in pixels, eps = 1 pixel)."""
    prob = workloads.random_problem(70, 90, C=3, seed=4)
    prm = dts.Params(lam=0.99, sigma_s=8.0, sigma_r=0.2, iterations=6, charbonnier_eps=1.0,
                     filter_kernel=dts.KERNEL_BOX)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm, charbonnier_eps=1.0, kernel=oracle.KERNEL_BOX)
    assert_close(z.cpu().numpy(), ref, prob.target, "charbonnier, box kernel")
    wl = workloads.make(1)
    p, q = wl.problems[0], wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes,
                     charbonnier_eps=1.0)
    z = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(p.guide, p.target, p.conf, prm, charbonnier_eps=1.0)
    assert_close(z.cpu().numpy(), ref, p.target, "charbonnier stereo 2880x1988")


@pytest.mark.parametrize("H,W", [(37, 53), (300, 257), (2300, 96)])
def test_solve_charbonnier_fixed_point_paper_eps(H, W):
    """The Charbonnier loss at the paper's eps = 0.001 with confidences in [0.1, 1], through the
    fixed point of Eq. 4 with the loss's weight at the current iterate (its steps are majorize-
    minimize steps, so FP32 and FP64 iterates do not part): the FP32 bound."""
    prob = workloads.random_problem(H, W, C=3, seed=H + 11 * W)
    prm = dts.Params(lam=0.99, sigma_s=8.0, sigma_r=0.2, iterations=10, update=dts.UPDATE_JACOBI,
                     charbonnier_eps=1e-3)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm, charbonnier_eps=1e-3)
    assert_close(z.cpu().numpy(), ref, prob.target, f"charbonnier fixed point {H}x{W}")


def test_solve_charbonnier_fixed_point_full_stereo_workload():
    """The stereo workload at full size (2880 x 1988, 20 iterations, confidences from the residual
    in [0.05, 1]) with the paper's stereo loss, eps = 0.001 pixel, through the fixed point of Eq. 4."""
    wl = workloads.make(1)
    p, q = wl.problems[0], wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes,
                     update=dts.UPDATE_JACOBI, charbonnier_eps=1e-3)
    z = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(p.guide, p.target, p.conf, prm, charbonnier_eps=1e-3)
    assert_close(z.cpu().numpy(), ref, p.target, "charbonnier fixed point stereo 2880x1988")


def test_solve_multispectral_reduced():
    """The 16-band multispectral generator at 2500 x 2500 (its full 10000 x 10000 size is timed
    by the bench): the 10-iteration solve against the oracle."""
    wl = workloads.make(4, H=2500, W=2500)
    p, q = wl.problems[0], wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
    z = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm)
    assert dts.dts_last_status() == 0
    ref = oracle_solve(p.guide, p.target, p.conf, prm)
    assert_close(z.cpu().numpy(), ref, p.target, "multispectral 2500x2500x16")


def test_solve_multispectral_full_size_constant_target():
    """The full 10000 x 10000 x 16 multispectral guide, in the launch configuration the bench
    times, with a constant target: every iterate stays that constant (a property the solve keeps
    at any size; the oracle cannot run this size)."""
    wl = workloads.make(4)
    p, q = wl.problems[0], wl.params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
    t = torch.full(p.target.shape, 0.625, device=dev())
    z = dts.dts_solve(to_dev(p.guide), t, to_dev(p.conf), prm)
    assert dts.dts_last_status() == 0
    assert float((z - 0.625).abs().max()) <= 1e-5


def multispectral_slice(H, W, seed=1004):
    """A slice of the 16-band multispectral generator at its full-size cell density (cells of about
    100 x 100 pixels): 10000 x 64 runs every vertical pass with the 10000-row plan of the full
    image, 64 x 10000 every horizontal pass with its 10000-column plan."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return workloads.multispectral_image(H, W, rng, bands=16, gy=max(1, H // 100), gx=max(1, W // 100))


@pytest.mark.parametrize("H,W", [(10000, 64), (64, 10000)])
@pytest.mark.parametrize("sdt", [torch.float32, torch.bfloat16])
def test_solve_multispectral_full_size_slices(H, W, sdt):
    """The multispectral solve (sigma_s 32, sigma_r 0.1, lambda 0.99, K = 10) on slices that run the
    full 10000 x 10000 image's launch plans, against the oracle element by element.  BF16 guide and
    target storage: within the FP32 bound of the oracle run on the same rounded inputs; from the
    oracle run on the unrounded inputs, no further than the rounding itself moves the oracle's
    solution plus that bound (with sigma_s / sigma_r = 320 the rounding of 16 guide bands moves the
    distances, and the solution, by a few percent of the target range)."""
    p = multispectral_slice(H, W)
    q = workloads.make(4, H=8, W=8).params
    prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=q.iterations, passes=q.passes)
    g, t = to_dev(p.guide, sdt), to_dev(p.target, sdt)
    z = dts.dts_solve(g, t, to_dev(p.conf), prm).cpu().numpy()
    assert dts.dts_last_status() == 0
    ref = oracle_solve(rounded(g), rounded(t), p.conf, prm)
    assert_close(z, ref, rounded(t), f"multispectral slice {H}x{W} on the stored inputs")
    if sdt != torch.float32:
        ref0 = oracle_solve(p.guide, p.target, p.conf, prm)
        rng0 = float(np.ptp(p.target))
        err = float(np.abs(z - ref0).max()) / rng0
        moved = float(np.abs(ref - ref0).max()) / rng0  # what the input rounding alone does
        assert err <= moved + TOL, f"bf16 storage: {err:.3e} of the range from the unrounded solve " \
                                   f"(rounding alone: {moved:.3e})"


# ---------------------------------------------------------------- streaming horizontal passes
# Rows of 1024 columns or more run on the streaming row kernel (row_stream_kernel: persistent CTAs,
# one row at a time, each row's input and distances copied into shared memory two rows ahead) when
# it takes them: a row length in whole 16-byte units (8 positions with FP16 distances) and two to
# sixteen warps' spans at 17 positions per thread (up to 8704 columns), else two to twelve at 33
# (up to 12672); other segment lengths and narrower rows as tuned plans, set here for row lengths
# no other test uses.  700 x 10000: four or five rows per CTA (both stages reused, both barrier
# parities); 12672: the widest row at 33; 12676 and 1101: not taken (the regular kernel runs);
# 1092 at 33: two warps, a ragged last segment; 8200 at 17: 16 warps; 1100 at 17: three warps.
# rows of any length: 1101, 1027, 2882 and 12038 end in 1-3 positions past their whole 16-byte units,
# which arrive by plain loads and leave by plain stores
STREAM_SHAPES = [(700, 10000, None), (3, 9000, None), (2, 12672, None), (2, 12676, None), (1500, 1100, 17),
                 (9, 1092, 33), (40, 2884, 33), (6, 1101, 33), (3, 8200, 17), (7, 1027, None), (4, 2882, 17),
                 (5, 12038, None)]


def stream_fits(W, items):
    nw = -(-(-(-W // items)) // 32)
    return 2 <= nw <= (12 if items == 33 else 16)


def stream_taken(W, items=None):
    """Whether the plan for W (a tuned segment length, or the default) runs the streaming kernel
    with FP32 distances."""
    if items is not None and stream_fits(W, items):
        return True
    return W >= 1024 and (stream_fits(W, 17) or stream_fits(W, 33))


def kernels_of(fn):
    dts.dts_profile(1)
    try:
        fn()
        torch.cuda.synchronize()
        return {r[0] for r in dts.dts_profile_read()}
    finally:
        dts.dts_profile(0)


@pytest.mark.parametrize("H,W,items", STREAM_SHAPES)
def test_filter_streaming_rows(H, W, items):
    if items is not None:
        dts.autotune_import("row %d %d\n" % (W, items))
    prob = workloads.random_problem(H, W, C=3, seed=H + 5 * W)
    prm = dts.Params(sigma_s=40.0, sigma_r=0.3, passes=3)
    g, src = to_dev(prob.guide), to_dev(prob.target)
    out = {}
    names = kernels_of(lambda: out.setdefault("z", dts.dts_filter(g, src, prm)))
    assert dts.dts_last_status() == 0
    assert ("row_stream_kernel" in names) == stream_taken(W, items), names
    ref = oracle.filter(prob.guide, prob.target, 40.0, 0.3, passes=3)
    assert_close(out["z"].cpu().numpy(), ref, prob.target, f"filter {H}x{W} items {items}")


# the data-term update in the streaming pass: Eq. 3, Eq. 4, the Charbonnier loss (both readings),
# BF16 and FP16 guide and target storage (each a kernel of its own), the support-weighted
# confidence (its chat plane), a caller's z_init; FP16 distances at 8200 and 8196 (a row of
# 16-byte units of FP32 but not of FP16: its last 4 distances by plain loads); rows that end past
# their whole 16-byte units (8202: two positions and distances, the update's last group one by
# one; 8203 with FP16 distances: three of each; 8201 with a BF16 target)
@pytest.mark.parametrize("variant", ["gd", "jacobi", "charbonnier_gd", "charbonnier_jacobi", "bf16", "f16target",
                                     "support", "zinit", "f16_8200", "f16_8196", "ragged_8202", "ragged_f16_8203",
                                     "ragged_bf16_8201"])
def test_solve_streaming_rows(variant):
    H, W = {"f16_8196": (24, 8196), "ragged_8202": (24, 8202), "ragged_f16_8203": (24, 8203),
            "ragged_bf16_8201": (24, 8201)}.get(variant, (24, 8200))
    prob = workloads.random_problem(H, W, C=3, seed=31 + len(variant))
    prm = dts.Params(lam=0.99, sigma_s=24.0, sigma_r=0.2, iterations=4)
    sdt, kw, z_init = torch.float32, {}, None
    if variant == "jacobi":
        prm.update = dts.UPDATE_JACOBI
    elif variant == "charbonnier_gd":
        prm.charbonnier_eps = 1.0
    elif variant == "charbonnier_jacobi":
        prm.update, prm.charbonnier_eps = dts.UPDATE_JACOBI, 1e-3
    elif variant in ("bf16", "ragged_bf16_8201"):
        sdt = torch.bfloat16
    elif variant == "f16target":
        sdt = torch.float16
    elif variant == "support":
        prm.conf_mode = dts.CONF_SUPPORT
    elif variant == "zinit":
        z_init = np.random.default_rng(5).random(prob.target.shape).astype(np.float32)
        kw["z_init"] = z_init.astype(np.float64)
    elif variant in ("f16_8200", "f16_8196", "ragged_f16_8203"):
        prm.dist_dtype = dts.F16
    g, t = to_dev(prob.guide, sdt), to_dev(prob.target, sdt)
    out = {}
    names = kernels_of(lambda: out.setdefault("z", dts.dts_solve(
        g, t, to_dev(prob.conf), prm, z_init=None if z_init is None else to_dev(z_init))))
    assert dts.dts_last_status() == 0
    assert "row_stream_kernel<update>" in names, names
    z = out["z"].cpu().numpy()
    if variant in ("f16_8200", "f16_8196", "ragged_f16_8203"):
        dX, dY = oracle.distances(prob.guide, 24.0, 0.2)
        ref = oracle.solve_d(dX.astype(np.float16).astype(np.float64), dY.astype(np.float16).astype(np.float64),
                             prob.target, prob.conf, lam=0.99, sigma_s=24.0, iterations=4)
    elif variant.startswith("charbonnier"):
        ref = oracle_solve(prob.guide, prob.target, prob.conf, prm, charbonnier_eps=prm.charbonnier_eps)
    else:
        ref = oracle_solve(rounded(g), rounded(t), prob.conf, prm, **kw)
    assert_close(z, ref, rounded(t), f"streaming rows, {variant}")


# ---------------------------------------------------------------- tall-column vertical passes
# Columns over 2176 rows run on persistent TMA-fed clusters (col_tall_kernel: 16 warps of 16, 32 or
# 40 rows per CTA, clusters of up to 16 CTAs: up to 10240 rows), taller ones on chains of CTAs
# (col_chain_kernel: 128-row chunks, 16 rows x 8 warps, by default; 256-row chunks, 16 x 16 and
# 32 x 8, as tuned shapes); the cluster kernel keeps tall columns for batched solves and as a
# tuned shape ((40, 16) in clusters of 7 here).  Each non-default shape is set through a tuned plan
# for a height no other test uses (tuned plans last for the process); cluster code -4 holds each
# column in a pair of clusters (top and bottom halves: 5 tiles of 512 rows as 3 + 3, 7 of 640 as
# 4 + 4, 16 of 640 as 8 + 8).  16384 rows is the tallest column.
@pytest.mark.parametrize("H,shape", [(2305, (16, 8, -1)), (2306, (16, 16, -1)), (2307, (32, 8, -1)),
                                     (2308, (16, 16, -2)), (2309, (32, 16, -2)), (2310, (40, 16, -2)),
                                     (4101, (40, 16, 7)), (2313, (32, 16, -4)), (4103, (40, 16, -4)),
                                     (10001, (40, 16, -4)), (10240, None), (12000, None), (16384, None)])
def test_filter_chain_and_cluster_shapes(H, shape):
    W = 70 if H < 10000 else 7
    if shape is not None:
        dts.autotune_import("col %d %d %d %d\n" % ((H,) + shape))
        assert ("col %d %d %d %d" % ((H,) + shape)) in dts.autotune_export()
    prob = workloads.random_problem(H, W, C=3, seed=H + W)
    prm = dts.Params(sigma_s=40.0, sigma_r=0.3, passes=3)
    out = dts.dts_filter(to_dev(prob.guide), to_dev(prob.target), prm)
    assert dts.dts_last_status() == 0
    ref = oracle.filter(prob.guide, prob.target, 40.0, 0.3, passes=3)
    assert_close(out.cpu().numpy(), ref, prob.target, f"filter {H}x{W} shape {shape}")


@pytest.mark.parametrize("variant", ["gd", "jacobi", "support", "cg"])
def test_solve_paired_tall_columns(variant):
    """Every kind of vertical pass (plain, the support sweep, the transposed pass of conjugate
    gradients) on the tall kernel with each column held by a pair of clusters."""
    H, W = 2316, 300
    dts.autotune_import("col %d 32 16 -4\n" % H)
    prob = workloads.random_problem(H, W, C=3, seed=79)
    prm = dts.Params(lam=0.99, sigma_s=24.0, sigma_r=0.2, iterations=3)
    if variant == "jacobi":
        prm.update = dts.UPDATE_JACOBI
    elif variant == "support":
        prm.conf_mode = dts.CONF_SUPPORT
    elif variant == "cg":
        prm.update = dts.UPDATE_CG
    out = {}
    names = kernels_of(lambda: out.setdefault("z", dts.dts_solve(to_dev(prob.guide), to_dev(prob.target),
                                                                 to_dev(prob.conf), prm)))
    assert dts.dts_last_status() == 0
    assert "col_tall_kernel" in names, names
    z = out["z"].cpu().numpy()
    if variant == "cg":
        ref = oracle.solve_cg(prob.guide, prob.target, prob.conf, lam=0.99, sigma_s=24.0, sigma_r=0.2,
                              iterations=3, passes=3)
    else:
        ref = oracle_solve(prob.guide, prob.target, prob.conf, prm)
    assert_close(z, ref, prob.target, f"paired tall columns, {variant}")


@pytest.mark.parametrize("update", [dts.UPDATE_GD, dts.UPDATE_JACOBI])
def test_solve_chained_columns_support_and_zinit(update):
    """Chained vertical passes inside the solve: the support-weighted confidence (its column sweep
    runs on the chain for any column over 256 rows) and a caller's z_init."""
    prob = workloads.random_problem(2600, 45, C=3, seed=26 + update)
    prm = dts.Params(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=4, update=update)
    z0 = np.random.default_rng(5).normal(size=prob.target.shape).astype(np.float32)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm, z_init=to_dev(z0))
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm, z_init=z0)
    assert_close(z.cpu().numpy(), ref, prob.target, "chain z_init")
    prm.conf_mode = dts.CONF_SUPPORT
    prm.update = dts.UPDATE_JACOBI
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    ref = oracle_solve(prob.guide, prob.target, prob.conf, prm)
    assert_close(z.cpu().numpy(), ref, prob.target, "chain support")
    assert dts.dts_last_status() == 0


# ---------------------------------------------------------------- confidence (Eq. 7)
@pytest.mark.parametrize("H,W,sdt", [(1, 1, torch.float32), (37, 53, torch.float32), (300, 517, torch.float32),
                                     (1200, 90, torch.bfloat16), (2100, 40, torch.float32)])
def test_confidence(H, W, sdt):
    """exp(-V / (2 sigma_c^2)), V = DT(t^2) - DT(t)^2, against the oracle on the same (rounded)
    target; c is in (0, 1], so the FP32 bound is absolute (1e-4, V computed from two FP32 means
    of values of order 1)."""
    prob = workloads.random_problem(H, W, C=3, seed=H + 5 * W)
    prm = dts.Params(sigma_s=10.0, sigma_r=0.2, passes=3)
    t = to_dev(prob.target, sdt)
    c = dts.dts_confidence(to_dev(prob.guide), t, prm, sigma_c=0.15)
    ref = oracle.confidence(prob.guide, rounded(t), 10.0, 0.2, sigma_c=0.15)
    assert float(np.abs(c.cpu().numpy() - ref).max()) <= 1e-4


def test_confidence_constant_target_is_one():
    """A constant target has zero variance.  In FP32 the two means of t = 3.25 and t^2 = 10.5625
    keep the constant to rounding through the segment exchanges, so V = DT(t^2) - DT(t)^2 is at
    most about 1e-5 and c >= exp(-1e-5 / (2 * 0.1^2)) ~ 1 - 5e-4."""
    prob = workloads.random_problem(120, 333, C=3, seed=9)
    c = dts.dts_confidence(to_dev(prob.guide), torch.full((120, 333), 3.25, device=dev()), dts.Params(), 0.1)
    assert float((c - 1.0).abs().max()) <= 1e-3


# ---------------------------------------------------------------- box kernel (Eq. 10's printed kernel)
def quantised_problem(H, W, seed, C=3):
    """Guide values on a 1/64 grid: with sigma_s / sigma_r = 32 every distance is an exact binary
    fraction on both sides, so the windows of the box kernel (a floating-point decision of which
    samples to average) are the same for the kernel and the oracle."""
    rng = np.random.default_rng(seed)
    p = workloads.random_problem(H, W, C=C, seed=seed)
    p.guide = (rng.integers(0, 65, (C, H, W)) / 64.0).astype(np.float32)
    return p


BOX = dict(sigma_s=8.0, sigma_r=0.25)


@pytest.mark.parametrize("H,W", [(1, 1), (1, 40), (29, 1), (7, 13), (33, 257), (300, 517), (1000, 77), (64, 2000),
                                 (2100, 40)])
def test_box_filter(H, W):
    prob = quantised_problem(H, W, seed=H * 13 + W)
    prm = dts.Params(passes=3, filter_kernel=dts.KERNEL_BOX, **BOX)
    out = dts.dts_filter(to_dev(prob.guide), to_dev(prob.target), prm)
    ref = oracle.box_filter(prob.guide, prob.target, passes=3, **BOX)
    assert_close(out.cpu().numpy(), ref, prob.target, f"box filter {H}x{W}")


@pytest.mark.parametrize("H,W,sigma_s", [(3, 8192, 8.0), (8192, 2, 8.0), (40, 300, 200.0), (300, 40, 200.0),
                                         (5, 700, 4000.0)])
def test_box_filter_long_lines_and_wide_windows(H, W, sigma_s):
    """Lines of the longest supported length, and windows wider than the line (sigma_s / sigma_r
    stays 32, so the windows are exact on both sides): the window ends are searched within
    floor(r) positions with a step count set by r."""
    prob = quantised_problem(H, W, seed=H * 7 + W)
    kw = dict(sigma_s=sigma_s, sigma_r=sigma_s / 32.0)
    prm = dts.Params(passes=3, filter_kernel=dts.KERNEL_BOX, **kw)
    out = dts.dts_filter(to_dev(prob.guide), to_dev(prob.target), prm)
    ref = oracle.box_filter(prob.guide, prob.target, passes=3, **kw)
    assert_close(out.cpu().numpy(), ref, prob.target, f"box filter {H}x{W} sigma_s={sigma_s}")


@pytest.mark.parametrize("update", [dts.UPDATE_GD, dts.UPDATE_JACOBI])
def test_box_solve(update):
    prob = quantised_problem(150, 211, seed=31 + update)
    prm = dts.Params(lam=0.9, iterations=6, update=update, filter_kernel=dts.KERNEL_BOX, **BOX)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), prm)
    ref = oracle.solve(prob.guide, prob.target, prob.conf, lam=0.9, iterations=6, update=update,
                       kernel=oracle.KERNEL_BOX, **BOX)
    assert_close(z.cpu().numpy(), ref, prob.target, f"box solve update={update}")


def test_box_kernel_limits():
    dev()
    g = torch.rand((3, 20, 30), device=dev())
    t = torch.rand((20, 30), device=dev())
    for kw in (dict(dist_dtype=dts.F16), dict(conf_mode=dts.CONF_SUPPORT)):
        with pytest.raises(RuntimeError):
            dts.dts_solve(g, t, t, dts.Params(filter_kernel=dts.KERNEL_BOX, **kw))
    with pytest.raises(RuntimeError):
        dts.dts_confidence(g, t, dts.Params(filter_kernel=dts.KERNEL_BOX), 0.1)


def test_host_pipeline_matches_direct_solves():
    """dts.HostPipeline (copies of neighbouring steps overlapping the solves, two device buffer
    sets, shapes changing between steps) gives the same results, bit for bit, as direct solves."""
    shapes = [(100, 130), (100, 130), (64, 80), (100, 130), (37, 51)]
    probs = [workloads.random_problem(H, W, C=3, seed=40 + i) for i, (H, W) in enumerate(shapes)]
    prm = dts.Params(lam=0.9, sigma_s=10.0, sigma_r=0.2, iterations=4)

    def solve_fn(din, dout):
        dts.dts_solve(din[0], din[1], din[2], prm, out=dout[0])

    hin = [[torch.from_numpy(x).pin_memory() for x in (p.guide, p.target, p.conf)] for p in probs]
    hout = [[torch.empty(p.target.shape, dtype=torch.float32).pin_memory()] for p in probs]
    dev()
    dts.HostPipeline(solve_fn).run(hin, hout)
    torch.cuda.synchronize()
    for p, (o,) in zip(probs, hout):
        ref = dts.dts_solve(to_dev(p.guide), to_dev(p.target), to_dev(p.conf), prm).cpu()
        assert torch.equal(o, ref)


def test_last_status_clean():
    dev()
    assert dts.dts_last_status() == 0
