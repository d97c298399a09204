"""Conjugate gradients on the objective of Eq. 2 (update = UPDATE_CG) through the C ABI:
the GPU iterates against the FP64 oracle's conjugate gradients on the same inputs, and
properties that hold at any size (the objective decreases, the gradient vanishes at the dense
minimiser, a constant target is kept).

Tolerance: max |gpu - oracle| <= 1e-4 * (max t - min t), the bound of the solver.  A product
M p takes 4N passes of FP32 rounding plus the elementwise step, and the dot products add in
FP64, so the iterates differ from the oracle's by rounding alone (observed at most 5e-7 of the
target range up to 40 iterations on these shapes).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1805_04590_gb300 import dts, workloads

pytestmark = pytest.mark.gpu

TOL = 1e-4
LAM, SIG_S, SIG_R = 0.99, 8.0, 0.2


def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch.device("cuda:0")


def to_dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev()).to(dtype)


def params(K, **kw):
    return dts.Params(lam=LAM, sigma_s=SIG_S, sigma_r=SIG_R, iterations=K, update=dts.UPDATE_CG, **kw)


def assert_close(z, ref, t, what=""):
    rng = float(np.ptp(t)) or 1.0
    err = float(np.abs(z - ref).max())
    assert err <= TOL * rng, f"{what}: max|gpu-oracle| = {err:.3e} > {TOL * rng:.3e}"


# one-CTA columns, columns of strip CTAs with 9- and 17-row segments, columns above the strip
# kernel's height (cluster kernel), long rows (up to 9000: 576-thread row CTAs), ragged widths
SHAPES = [(37, 53), (130, 300), (300, 257), (1100, 96), (2300, 70), (70, 5000), (20, 9000)]


@pytest.mark.parametrize("H,W", SHAPES)
@pytest.mark.parametrize("K", [0, 1, 3, 10])
def test_cg_matches_oracle(H, W, K):
    prob = workloads.random_problem(H, W, seed=H + W)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), params(K))
    torch.cuda.synchronize()
    assert dts.dts_last_status() == 0
    ref = oracle.solve_cg(prob.guide, prob.target, prob.conf, lam=LAM, sigma_s=SIG_S, sigma_r=SIG_R, iterations=K)
    assert_close(z.cpu().numpy(), ref, prob.target, f"{H}x{W} K={K}")


@pytest.mark.parametrize("H,W", [(1, 1), (1, 23), (29, 1), (2, 2), (3, 700)])
def test_cg_degenerate_shapes(H, W):
    """Lines of one position (the passes are the identity there) and very short lines."""
    prob = workloads.random_problem(H, W, seed=3 * H + W)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), params(4))
    torch.cuda.synchronize()
    assert dts.dts_last_status() == 0
    ref = oracle.solve_cg(prob.guide, prob.target, prob.conf, lam=LAM, sigma_s=SIG_S, sigma_r=SIG_R, iterations=4)
    assert_close(z.cpu().numpy(), ref, prob.target, f"{H}x{W}")


def test_cg_first_step_uses_the_transposed_filter():
    """One step from z_0 = t: r_0 = 2 C t - M t involves A^T.  The same step with A in place of
    A^T (a plausible slip) is far from the GPU result, so the check can tell them apart."""
    prob = workloads.random_problem(90, 140, seed=3)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf), params(1)).cpu().numpy()
    dX, dY = oracle.distances(prob.guide, SIG_S, SIG_R)
    _, a = oracle.schedule(SIG_S, 3)
    t, c = prob.target.astype(np.float64), prob.conf.astype(np.float64)
    ref = oracle.solve_cg_d(dX, dY, t, c, lam=LAM, sigma_s=SIG_S, iterations=1)
    assert_close(z, ref, t, "K=1")
    A = lambda v: oracle.filter_d(dX, dY, a, v)
    v = t - A(t)
    r0 = 2 * c * t - (LAM * (v - A(v)) + 2 * c * t)  # A in place of A^T
    Mr = LAM * ((r0 - A(r0)) - A(r0 - A(r0))) + 2 * c * r0
    wrong = t + (np.sum(r0 * r0) / np.sum(r0 * Mr)) * r0
    assert np.abs(z - wrong).max() > 100 * TOL * np.ptp(t)


def test_cg_initial_guess_and_16bit_storage():
    """z_init, a BF16 target and FP16 distance planes: against the oracle on the same rounded
    inputs (its FP64 distances rounded to FP16)."""
    prob = workloads.random_problem(160, 230, seed=21)
    z0 = np.asarray(prob.target * 0.5 + 0.25, dtype=np.float32)
    tb = to_dev(prob.target, torch.bfloat16)
    z = dts.dts_solve(to_dev(prob.guide), tb, to_dev(prob.conf), params(6, dist_dtype=dts.F16),
                      z_init=to_dev(z0)).cpu().numpy()
    dX, dY = oracle.distances(prob.guide, SIG_S, SIG_R)
    dX = dX.astype(np.float16).astype(np.float64)
    dY = dY.astype(np.float16).astype(np.float64)
    t = tb.float().cpu().numpy().astype(np.float64)
    ref = oracle.solve_cg_d(dX, dY, t, prob.conf, lam=LAM, sigma_s=SIG_S, iterations=6, z_init=z0)
    assert_close(z, ref, t, "z_init, bf16 target, fp16 distances")


def dense_filter_matrix(dX, dY, a):
    n = dX.size
    E = np.eye(n).reshape(n, *dX.shape)
    return np.stack([oracle.filter_d(dX, dY, a, e).ravel() for e in E], axis=1)


def test_cg_reaches_the_dense_minimiser():
    """Enough steps reach the solution of (lambda (I - A)^T (I - A) + 2C) z = 2 C t, solved
    densely; the paper's update of Eq. 3 after as many iterations has a larger objective."""
    prob = workloads.random_problem(18, 24, seed=8)
    dX, dY = oracle.distances(prob.guide, SIG_S, SIG_R)
    _, a = oracle.schedule(SIG_S, 3)
    A = dense_filter_matrix(dX, dY, a)
    n = A.shape[0]
    t, c = prob.target.astype(np.float64).ravel(), prob.conf.astype(np.float64).ravel()
    B = np.eye(n) - A
    M = LAM * B.T @ B + 2 * np.diag(c)
    zs = np.linalg.solve(M, 2 * c * t)
    g, tt, cc = to_dev(prob.guide), to_dev(prob.target), to_dev(prob.conf)
    z = dts.dts_solve(g, tt, cc, params(150)).cpu().numpy().astype(np.float64).ravel()
    assert np.abs(z - zs).max() <= TOL * np.ptp(t)
    F = lambda v: 0.5 * LAM * np.sum((B @ v) ** 2) + np.sum(c * (v - t) ** 2)
    zgd = dts.dts_solve(g, tt, cc, dts.Params(lam=LAM, sigma_s=SIG_S, sigma_r=SIG_R, iterations=150))
    assert F(z) < F(zgd.cpu().numpy().astype(np.float64).ravel())


def test_cg_keeps_a_constant_target():
    prob = workloads.random_problem(120, 170, seed=9)
    t = np.full(prob.target.shape, 0.37, np.float32)
    z = dts.dts_solve(to_dev(prob.guide), to_dev(t), to_dev(prob.conf), params(10)).cpu().numpy()
    assert np.abs(z - 0.37).max() <= 1e-5


def test_cg_batched_matches_oracle():
    wl = workloads.workload_batched(seed=31, n=5, hmin=17, hmax=300, wmin=9, wmax=400)
    g = [to_dev(p.guide) for p in wl.problems]
    t = [to_dev(p.target) for p in wl.problems]
    c = [to_dev(p.conf) for p in wl.problems]
    outs = dts.dts_solve_batched(g, t, c, params(5))
    torch.cuda.synchronize()
    assert dts.dts_last_status() == 0
    for i, p in enumerate(wl.problems):
        ref = oracle.solve_cg(p.guide, p.target, p.conf, lam=LAM, sigma_s=SIG_S, sigma_r=SIG_R, iterations=5)
        assert_close(outs[i].cpu().numpy(), ref, p.target, f"image {i}")


def objective(g, t, c, z, prm):
    """F(z) of Eq. 2 in FP64 from the GPU filter: lambda/2 |z - A z|^2 + sum c (z - t)^2."""
    Az = dts.dts_filter(g, z, prm).double()
    zd = z.double()
    return float(0.5 * prm.lam * ((zd - Az) ** 2).sum() + (c.double() * (zd - t.double()) ** 2).sum())


def test_cg_objective_decreases_on_the_full_stereo_workload():
    """At 2880 x 1988: each further step lowers the objective (CG minimises the energy norm of
    the error over a growing space), up to FP32 rounding of the objective itself."""
    wl = workloads.make(1)
    p = wl.problems[0]
    q = wl.params
    g, t, c = to_dev(p.guide), to_dev(p.target), to_dev(p.conf)
    vals = []
    for K in (0, 1, 2, 5, 10, 20):
        prm = dts.Params(lam=q.lam, sigma_s=q.sigma_s, sigma_r=q.sigma_r, iterations=K, passes=q.passes,
                         update=dts.UPDATE_CG)
        z = dts.dts_solve(g, t, c, prm)
        torch.cuda.synchronize()
        assert dts.dts_last_status() == 0
        vals.append(objective(g, t, c, z, prm))
    for a, b in zip(vals, vals[1:]):
        assert b <= a * (1 + 1e-5), vals
    assert vals[-1] < vals[0], vals
