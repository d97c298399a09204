"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: explicit
sum expansions of the recurrences, a dense matrix built from products of
weights, closed forms for a uniform guide, invariants of the normalised
filter, a direct linear solve of the fixed point of Eq. 4, finite
differences and an independent autograd restatement.  The paper prints no
worked numeric example and its Tables 1-2 need datasets that are absent, so
those values stay unpinned.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_1805_04590_gb300 import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ---------------------------------------------------------------- helpers
def causal_matrix(d, a):
    """Explicit expansion J[n] = (prod_{m=1..n} w_m) x[0] + sum_{j=1..n} (1-w_j) prod_{m=j+1..n} w_m x[j]."""
    n = len(d)
    w = [a ** d[j] for j in range(n)]
    L = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1):
            coef = 1.0 if j == 0 else 1.0 - w[j]
            for m in range(j + 1, i + 1):
                coef *= w[m]
            L[i, j] = coef
    return L


def anticausal_matrix(d, a):
    """Explicit expansion of K[i] = (1-w'_i) x[i] + w'_i K[i+1], w'_i = a^d[i+1]."""
    n = len(d)
    wp = [a ** d[j + 1] if j + 1 < n else 0.0 for j in range(n)]
    R = np.zeros((n, n))
    for i in range(n):
        for j in range(i, n):
            coef = 1.0 if j == n - 1 else 1.0 - wp[j]
            for m in range(i, j):
                coef *= wp[m]
            R[i, j] = coef
    return R


def dense_filter_matrix(dX, dY, a_list):
    """A = V_N H_N ... V_1 H_1 on the row-major flattened image, each pass the
    product (anti-causal matrix) x (causal matrix) of its lines."""
    H, W = dX.shape
    n = H * W
    M = np.eye(n)
    for a in a_list:
        Hm = np.zeros((n, n))
        for y in range(H):
            P = anticausal_matrix(dX[y], a) @ causal_matrix(dX[y], a)
            idx = y * W + np.arange(W)
            Hm[np.ix_(idx, idx)] = P
        Vm = np.zeros((n, n))
        for x in range(W):
            P = anticausal_matrix(dY[:, x], a) @ causal_matrix(dY[:, x], a)
            idx = np.arange(H) * W + x
            Vm[np.ix_(idx, idx)] = P
        M = Vm @ (Hm @ M)
    return M


def oracle_filter_matrix(dX, dY, a_list):
    H, W = dX.shape
    n = H * W
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = oracle.filter_d(dX, dY, a_list, e.reshape(H, W)).reshape(-1)
    return M


def rand_guide(rng, C, H, W):
    return rng.random((C, H, W))


# ---------------------------------------------------------------- recurrences
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8])
def test_sweeps_match_sum_expansion(n):
    rng = np.random.default_rng(n)
    for _ in range(5):
        x = rng.normal(size=n)
        d = 1.0 + 5.0 * rng.random(n)
        a = rng.uniform(0.2, 0.95)
        np.testing.assert_allclose(oracle.causal(x, d, a), causal_matrix(d, a) @ x, rtol=0, atol=1e-15)
        np.testing.assert_allclose(oracle.anticausal(x, d, a), anticausal_matrix(d, a) @ x, rtol=0, atol=1e-15)


def test_hand_worked_pass():
    g = json.load(open(os.path.join(GOLDEN, "sweep_hand.json")))
    J = oracle.causal(g["x"], g["d"], g["a"])
    assert J.tolist() == g["causal"]
    K = oracle.anticausal(J, g["d"], g["a"])
    assert K.tolist() == g["pass"]
    u = oracle.row_pass(np.array([g["x"]]), np.array([g["d"]]), g["a"])
    assert u[0].tolist() == g["pass"]


@pytest.mark.parametrize("a", [0.3, 0.8, 0.95])
def test_uniform_guide_impulse_response(a):
    """d = 1 everywhere: causal then anti-causal on an impulse equals
    (1-a)/(1+a) a^|n| away from the borders; sum 1, variance 2a/(1-a)^2."""
    n = 1201
    c = n // 2
    x = np.zeros(n)
    x[c] = 1.0
    d = np.ones(n)
    y = oracle.anticausal(oracle.causal(x, d, a), d, a)
    k = np.arange(n) - c
    expect = (1 - a) / (1 + a) * a ** np.abs(k)
    np.testing.assert_allclose(y, expect, rtol=0, atol=1e-13)
    assert abs(y.sum() - 1.0) < 1e-12
    var = (y * k * k).sum()
    assert abs(var - 2 * a / (1 - a) ** 2) < 1e-9 * max(1.0, var)


def test_schedule_variance_and_halving():
    for sigma_s in (1.0, 8.0, 64.0, 320.0):
        for N in (1, 2, 3, 5):
            sig, a = oracle.schedule(sigma_s, N)
            assert abs((sig ** 2).sum() - sigma_s ** 2) < 1e-12 * sigma_s ** 2
            if N > 1:
                np.testing.assert_allclose(sig[:-1] / sig[1:], 2.0, rtol=1e-14)
            np.testing.assert_allclose(np.log(a) * sig, -math.sqrt(2.0), rtol=1e-14)
    sig, _ = oracle.schedule(5.0, 1)
    assert abs(sig[0] - 5.0) < 1e-14


def test_recursive_filter_variance_matches_sigma():
    """The feedback a = exp(-sqrt(2)/sigma) makes the 1-D pass variance
    2a/(1-a)^2 approach sigma^2 for large sigma (G&O's design rule)."""
    for s in (20.0, 80.0, 320.0):
        a = math.exp(-math.sqrt(2) / s)
        assert abs(2 * a / (1 - a) ** 2 / s ** 2 - 1) < 2.0 / s ** 2 + 1e-12


# ---------------------------------------------------------------- distances
def test_distances_hand_values():
    I = np.array([[[0.0, 0.5, 0.25], [1.0, 1.0, 0.0]],
                  [[0.0, 0.0, 0.5], [0.0, 0.25, 0.5]]])
    dX, dY = oracle.distances(I, sigma_s=2.0, sigma_r=1.0, norm=oracle.NORM_L1)
    np.testing.assert_allclose(dX, [[1, 2.0, 2.5], [1, 1.5, 3.5]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(dY, [[1, 1, 1], [3.0, 2.5, 1.5]], rtol=0, atol=1e-15)
    dX2, dY2 = oracle.distances(I, sigma_s=2.0, sigma_r=1.0, norm=oracle.NORM_L2)
    # sqrt(1 + 4 * sum of squared differences)
    np.testing.assert_allclose(dX2, [[1, math.sqrt(2.0), math.sqrt(1 + 4 * (0.0625 + 0.25))],
                                     [1, math.sqrt(1 + 4 * 0.0625), math.sqrt(1 + 4 * (1 + 0.0625))]], atol=1e-15)
    np.testing.assert_allclose(dY2, [[1, 1, 1], [math.sqrt(5.0), math.sqrt(1 + 4 * (0.25 + 0.0625)),
                                                 math.sqrt(1 + 4 * 0.0625)]], atol=1e-15)


def test_constant_guide_unit_distances():
    I = np.full((4, 5, 6), 0.37)
    dX, dY = oracle.distances(I, 8.0, 0.2)
    assert (dX == 1).all() and (dY == 1).all()


# ---------------------------------------------------------------- filter
@pytest.mark.parametrize("H,W,N", [(5, 7, 3), (4, 4, 1), (1, 6, 2), (6, 1, 2), (3, 5, 2)])
def test_filter_equals_dense_product(H, W, N):
    rng = np.random.default_rng(100 + H * W + N)
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 6.0, 0.5)
    _, a = oracle.schedule(6.0, N)
    Ad = dense_filter_matrix(dX, dY, a)
    Ao = oracle_filter_matrix(dX, dY, a)
    np.testing.assert_allclose(Ao, Ad, rtol=0, atol=1e-13)


def test_filter_row_stochastic_and_constant_preserving():
    rng = np.random.default_rng(7)
    I = rand_guide(rng, 3, 9, 11)
    dX, dY = oracle.distances(I, 8.0, 0.2)
    _, a = oracle.schedule(8.0, 3)
    A = oracle_filter_matrix(dX, dY, a)
    assert (A >= 0).all()
    np.testing.assert_allclose(A.sum(1), 1.0, rtol=0, atol=1e-13)
    c = oracle.filter_d(dX, dY, a, np.full((9, 11), -3.25))
    np.testing.assert_allclose(c, -3.25, rtol=0, atol=1e-13)


def test_degenerate_shapes():
    rng = np.random.default_rng(3)
    # 1 x 1: the filter is the identity
    I = rand_guide(rng, 2, 1, 1)
    assert oracle.filter(I, np.array([[2.5]]), 8.0, 0.2)[0, 0] == 2.5
    # H = 1: only the horizontal passes act
    I = rand_guide(rng, 3, 1, 9)
    u = rng.normal(size=(1, 9))
    dX, dY = oracle.distances(I, 8.0, 0.2)
    _, a = oracle.schedule(8.0, 3)
    ref = u.copy()
    for ai in a:
        ref = oracle.row_pass(ref, dX, ai)
    np.testing.assert_allclose(oracle.filter_d(dX, dY, a, u), ref, atol=1e-15)
    # W = 1: only the vertical passes act
    I = rand_guide(rng, 3, 9, 1)
    u = rng.normal(size=(9, 1))
    dX, dY = oracle.distances(I, 8.0, 0.2)
    ref = u.copy()
    for ai in a:
        ref = oracle.col_pass(ref, dY, ai)
    np.testing.assert_allclose(oracle.filter_d(dX, dY, a, u), ref, atol=1e-15)


def test_step_edge_leakage_bound():
    """Across a colour step of height h the recursive weight is a^(1 + sigma_s h / sigma_r):
    each pass moves at most twice that fraction across the edge."""
    W = 80
    I = np.zeros((1, 1, W))
    I[0, 0, W // 2:] = 1.0
    u = np.zeros((1, W))
    u[0, :W // 2] = 1.0
    sigma_s, sigma_r = 8.0, 0.2
    dX, dY = oracle.distances(I, sigma_s, sigma_r)
    assert dX[0, W // 2] == 1 + sigma_s / sigma_r
    _, a = oracle.schedule(sigma_s, 3)
    out = oracle.filter_d(dX, dY, a, u)
    bound = sum(2 * ai ** (1 + sigma_s / sigma_r) for ai in a)
    assert np.abs(out[0, :W // 2] - 1.0).max() <= bound
    assert np.abs(out[0, W // 2:]).max() <= bound
    assert bound < 1e-3
    # two-pixel case in closed form: J1 = w x0 with w = a^(1 + sigma_s h / sigma_r)
    J = oracle.causal([1.0, 0.0], [1.0, 1 + sigma_s / sigma_r], a[0])
    assert abs(J[1] - a[0] ** (1 + sigma_s / sigma_r)) < 1e-18


# ---------------------------------------------------------------- solver
def _small(H=6, W=7, seed=11):
    rng = np.random.default_rng(seed)
    I = rand_guide(rng, 3, H, W)
    t = rng.normal(size=(H, W))
    c = rng.uniform(0.2, 1.0, (H, W))
    return I, t, c


def test_solve_with_zero_confidence_is_the_filter():
    I, t, _ = _small()
    c = np.zeros_like(t)
    zf = oracle.filter(I, t, 8.0, 0.2)
    zj = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=1, update=oracle.UPDATE_JACOBI)
    zg = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=1, step=1.0)
    np.testing.assert_allclose(zj, zf, atol=1e-14)
    np.testing.assert_allclose(zg, zf, atol=1e-14)


def test_one_step_matches_dense_update():
    I, t, c = _small()
    z0 = np.random.default_rng(5).normal(size=t.shape)
    dX, dY = oracle.distances(I, 8.0, 0.2)
    _, a = oracle.schedule(8.0, 3)
    A = dense_filter_matrix(dX, dY, a)
    zbar = (A @ z0.reshape(-1)).reshape(t.shape)
    lam, eta = 0.7, 0.99
    gd = z0 - eta * (lam * (z0 - zbar) + c * (z0 - t))
    jac = (lam * zbar + c * t) / (lam + c)
    z1 = oracle.solve(I, t, c, lam=lam, sigma_s=8.0, sigma_r=0.2, step=eta, iterations=1, z_init=z0)
    np.testing.assert_allclose(z1, gd, atol=1e-13)
    z1 = oracle.solve(I, t, c, lam=lam, sigma_s=8.0, sigma_r=0.2, iterations=1, z_init=z0,
                      update=oracle.UPDATE_JACOBI)
    np.testing.assert_allclose(z1, jac, atol=1e-13)


@pytest.mark.parametrize("update", [oracle.UPDATE_GD, oracle.UPDATE_JACOBI])
def test_iterations_converge_to_dense_fixed_point(update):
    """The update of Eq. 3 (step 0.99) and its fixed point Eq. 4 both converge
    to the solution of (lambda (I - A) + C) z = C t."""
    I, t, c = _small(5, 6, 21)
    lam = 1.0
    dX, dY = oracle.distances(I, 8.0, 0.2)
    _, a = oracle.schedule(8.0, 3)
    A = dense_filter_matrix(dX, dY, a)
    n = t.size
    M = lam * (np.eye(n) - A) + np.diag(c.reshape(-1))
    zstar = np.linalg.solve(M, (c * t).reshape(-1)).reshape(t.shape)
    z = oracle.solve(I, t, c, lam=lam, sigma_s=8.0, sigma_r=0.2, iterations=4000, update=update)
    np.testing.assert_allclose(z, zstar, rtol=0, atol=1e-10)


def test_constant_target_is_a_fixed_point_and_lambda_zero():
    I, t, c = _small()
    t0 = np.full_like(t, 0.625)
    for upd in (oracle.UPDATE_GD, oracle.UPDATE_JACOBI):
        z = oracle.solve(I, t0, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=7, update=upd)
        np.testing.assert_allclose(z, 0.625, atol=1e-14)
    z0 = np.random.default_rng(1).normal(size=t.shape)
    z = oracle.solve(I, t, c, lam=0.0, sigma_s=8.0, sigma_r=0.2, iterations=1, update=oracle.UPDATE_JACOBI,
                     z_init=z0)
    np.testing.assert_allclose(z, t, atol=1e-15)


def test_zero_iterations_returns_start():
    I, t, c = _small()
    z = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=0)
    np.testing.assert_array_equal(z, t)


def test_checkpoints_are_the_iterates():
    I, t, c = _small()
    z, ck = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=3, checkpoints=True)
    np.testing.assert_array_equal(ck[0], t)
    z1 = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=1)
    np.testing.assert_allclose(ck[1], z1, atol=1e-15)
    z2 = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=1, z_init=ck[2])
    np.testing.assert_allclose(z, z2, atol=1e-15)


# ---------------------------------------------------------------- support weighting
def test_support_brute_force_and_flat_limit():
    rng = np.random.default_rng(9)
    H, W, sigma_s = 4, 5, 6.0
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, sigma_s, 0.5)
    S, sf = oracle.support(dX, dY, sigma_s)
    a = math.exp(-math.sqrt(2) / sigma_s)
    cum_x = np.concatenate([np.zeros((H, 1)), np.cumsum(dX[:, 1:], 1)], 1)
    cum_y = np.concatenate([np.zeros((1, W)), np.cumsum(dY[1:], 0)], 0)
    Sb = np.zeros((H, W))
    for y in range(H):
        for x in range(W):
            tot = 0.0
            for yy in range(H):
                wy = a ** abs(cum_y[y, x] - cum_y[yy, x])
                s_row = sum(a ** abs(cum_x[yy, x] - cum_x[yy, xx]) for xx in range(W))
                tot += wy * s_row
            Sb[y, x] = tot
    np.testing.assert_allclose(S, Sb, rtol=1e-12)
    assert abs(sf - ((1 + a) / (1 - a)) ** 2) < 1e-12 * sf
    # flat guide: the interior of a large image reaches the unbounded value
    Hh = Ww = 301
    S2, sf2 = oracle.support(np.ones((Hh, Ww)), np.ones((Hh, Ww)), 4.0)
    assert abs(S2[150, 150] / sf2 - 1) < 1e-12


def test_support_mode_equals_plain_on_scaled_confidence():
    I, t, c = _small()
    dX, dY = oracle.distances(I, 8.0, 0.2)
    S, sf = oracle.support(dX, dY, 8.0)
    chat = c * sf / S
    z_s = oracle.solve(I, t, c, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=4, update=oracle.UPDATE_JACOBI,
                       conf_mode=oracle.CONF_SUPPORT)
    z_p = oracle.solve(I, t, chat, lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=4, update=oracle.UPDATE_JACOBI)
    np.testing.assert_allclose(z_s, z_p, atol=1e-14)


def test_support_gradient_step_is_limited_per_pixel():
    """Reading of the support weighting for the gradient step: where the weighted confidence chat
    is large the step at pixel i is min(eta, 1 / (lambda + chat_i)).  One step from z0 against
    that update written out, on a case where the limit holds at some pixels and not at others."""
    rng = np.random.default_rng(23)
    H, W, sigma_s, sigma_r = 9, 11, 6.0, 0.3
    I = rand_guide(rng, 3, H, W)
    t, z0 = rng.random((H, W)), rng.random((H, W))
    c = 10.0 ** rng.uniform(-3.0, 0.3, (H, W))
    lam, eta = 0.5, 0.99
    dX, dY = oracle.distances(I, sigma_s, sigma_r)
    S, sf = oracle.support(dX, dY, sigma_s)
    chat = c * sf / S
    _, a = oracle.schedule(sigma_s, 3)
    e = np.minimum(eta, 1.0 / (lam + chat))
    assert (e < eta).any() and (e == eta).any()
    want = z0 - e * (lam * (z0 - oracle.filter_d(dX, dY, a, z0)) + chat * (z0 - t))
    got = oracle.solve(I, t, c, lam=lam, sigma_s=sigma_s, sigma_r=sigma_r, step=eta, iterations=1,
                       update=oracle.UPDATE_GD, conf_mode=oracle.CONF_SUPPORT, z_init=z0)
    np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


# ---------------------------------------------------------------- reverse mode
def test_filter_adjoint_dot_product_and_dense_transpose():
    rng = np.random.default_rng(17)
    H, W = 6, 5
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 8.0, 0.2)
    _, a = oracle.schedule(8.0, 3)
    u = rng.normal(size=(H, W))
    v = rng.normal(size=(H, W))
    Au = oracle.filter_d(dX, dY, a, u)
    ATv, _, _ = oracle.filter_adjoint(dX, dY, a, u, v)
    assert abs((Au * v).sum() - (u * ATv).sum()) < 1e-12
    A = dense_filter_matrix(dX, dY, a)
    np.testing.assert_allclose(ATv.reshape(-1), A.T @ v.reshape(-1), atol=1e-13)


def _objective(I, t, c, gz, z0=None, **kw):
    return float((oracle.solve(I, t, c, z_init=z0, **kw) * gz).sum())


# the last case: the gradient step with the Charbonnier target loss (eps where the loss is smooth
# on the scale of the difference step)
@pytest.mark.parametrize("update,norm,eps", [(oracle.UPDATE_GD, oracle.NORM_L1, 0.0),
                                             (oracle.UPDATE_JACOBI, oracle.NORM_L1, 0.0),
                                             (oracle.UPDATE_GD, oracle.NORM_L2, 0.0),
                                             (oracle.UPDATE_GD, oracle.NORM_L1, 0.3),
                                             (oracle.UPDATE_JACOBI, oracle.NORM_L1, 0.3),
                                             (oracle.UPDATE_JACOBI, oracle.NORM_L2, 0.05)])
def test_backward_matches_central_differences(update, norm, eps):
    rng = np.random.default_rng(23 + update + 2 * norm)
    C, H, W = 2, 5, 6
    I = rand_guide(rng, C, H, W)
    t = rng.normal(size=(H, W))
    c = rng.uniform(0.2, 1.0, (H, W))
    gz = rng.normal(size=(H, W))
    kw = dict(lam=0.9, sigma_s=4.0, sigma_r=0.5, iterations=3, update=update, norm=norm, charbonnier_eps=eps)
    g = oracle.solve_backward(I, t, c, gz, **kw)
    h = 1e-6
    for name, arr in (("t", t), ("c", c), ("guide", I)):
        flat = arr.reshape(-1)
        for idx in rng.choice(flat.size, 8, replace=False):
            old = flat[idx]
            flat[idx] = old + h
            fp = _objective(I, t, c, gz, **kw)
            flat[idx] = old - h
            fm = _objective(I, t, c, gz, **kw)
            flat[idx] = old
            fd = (fp - fm) / (2 * h)
            an = g[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-6 * max(1.0, abs(fd)), (name, idx, fd, an)
    z0 = rng.normal(size=(H, W))
    g0 = oracle.solve_backward(I, t, c, gz, z_init=z0, **kw)
    flat = z0.reshape(-1)
    for idx in rng.choice(flat.size, 5, replace=False):
        old = flat[idx]
        flat[idx] = old + h
        fp = _objective(I, t, c, gz, z0=z0, **kw)
        flat[idx] = old - h
        fm = _objective(I, t, c, gz, z0=z0, **kw)
        flat[idx] = old
        assert abs((fp - fm) / (2 * h) - g0["z_init"].reshape(-1)[idx]) <= 1e-6


@pytest.mark.parametrize("update,norm", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_backward_matches_autograd_restatement(update, norm):
    torch = pytest.importorskip("torch")
    from tests import autograd_ref as ref
    rng = np.random.default_rng(31 + update + 2 * norm)
    C, H, W = 3, 6, 7
    I = rand_guide(rng, C, H, W)
    t = rng.normal(size=(H, W))
    c = rng.uniform(0.2, 1.0, (H, W))
    gz = rng.normal(size=(H, W))
    kw = dict(lam=0.8, sigma_s=5.0, sigma_r=0.4, step=0.99, iterations=3, passes=3, norm=norm, update=update)
    It = torch.tensor(I, requires_grad=True)
    tt = torch.tensor(t, requires_grad=True)
    ct = torch.tensor(c, requires_grad=True)
    z = ref.solve(It, tt, ct, **kw)
    np.testing.assert_allclose(z.detach().numpy(), oracle.solve(I, t, c, **kw), atol=1e-12)
    (z * torch.tensor(gz)).sum().backward()
    g = oracle.solve_backward(I, t, c, gz, **kw)
    np.testing.assert_allclose(g["t"], tt.grad.numpy(), atol=1e-10)
    np.testing.assert_allclose(g["c"], ct.grad.numpy(), atol=1e-10)
    np.testing.assert_allclose(g["guide"], It.grad.numpy(), atol=1e-10)


def test_workload_generators_are_seeded():
    a = workloads.make(0)
    b = workloads.make(0)
    p, q = a.problems[0], b.problems[0]
    assert p.guide.shape == (3, 256, 256) and p.guide.dtype == np.float32
    np.testing.assert_array_equal(p.guide, q.guide)
    np.testing.assert_array_equal(p.target, q.target)
    assert 0.2 <= p.conf.min() and p.conf.max() <= 1.0
    assert a.params.sigma_s == 8.0 and a.params.iterations == 10


# ---------------------------------------------------------------- confidence (Eq. 7)
def test_confidence_equals_dense_variance():
    """c = exp(-V / (2 sigma_c^2)) with V_i = sum_j A_ij t_j^2 - (sum_j A_ij t_j)^2 computed from
    the dense filter matrix (built from weight products, independent of the oracle's sweeps)."""
    rng = np.random.default_rng(71)
    H, W = 5, 6
    I = rand_guide(rng, 3, H, W)
    t = rng.normal(size=(H, W))
    dX, dY = oracle.distances(I, 6.0, 0.4)
    _, a = oracle.schedule(6.0, 3)
    A = dense_filter_matrix(dX, dY, a)
    tf = t.ravel()
    V = A @ (tf * tf) - (A @ tf) ** 2
    ref = np.exp(-np.maximum(V, 0.0) / (2 * 0.3 ** 2)).reshape(H, W)
    got = oracle.confidence_d(dX, dY, a, t, 0.3)
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13)


def test_confidence_properties():
    rng = np.random.default_rng(72)
    I = rand_guide(rng, 3, 12, 15)
    # a constant target has zero variance: full confidence everywhere
    c = oracle.confidence(I, np.full((12, 15), 0.7), 8.0, 0.2, sigma_c=0.1)
    np.testing.assert_allclose(c, 1.0, rtol=0, atol=1e-12)
    # the variance is non-negative (Jensen: A is non-negative and row-stochastic), so c <= 1,
    # and a larger sigma_c never lowers the confidence
    t = rng.normal(size=(12, 15))
    c1 = oracle.confidence(I, t, 8.0, 0.2, sigma_c=0.2)
    c2 = oracle.confidence(I, t, 8.0, 0.2, sigma_c=0.5)
    assert (c1 <= 1.0).all() and (c1 > 0.0).all() and (c2 >= c1).all()
    # two flat regions split by a strong guide edge: the variance stays near 0 away from it
    G = np.zeros((1, 8, 16))
    G[:, :, 8:] = 1.0
    tt = np.where(np.arange(16) < 8, 0.0, 1.0)[None, :].repeat(8, 0)
    c = oracle.confidence(G, tt, 8.0, 0.05, sigma_c=0.1)
    assert c[:, :4].min() > 0.999 and c[:, 12:].min() > 0.999


# ---------------------------------------------------------------- box-kernel filter (Eq. 10's printed kernel)
def box_pass_dense(d_line, r):
    """Row-normalised 0/1 matrix of one line: W_nm = 1 if |ct_n - ct_m| <= r, ct a cumulative sum
    of the distances (numpy cumsum, independent of the oracle's loop)."""
    ct = np.concatenate([[0.0], np.cumsum(d_line[1:])])
    Wm = (np.abs(ct[:, None] - ct[None, :]) <= r).astype(float)
    return Wm / Wm.sum(1, keepdims=True)


@pytest.mark.parametrize("H,W,N", [(5, 7, 3), (1, 9, 2), (8, 1, 2), (6, 6, 1)])
def test_box_filter_equals_dense_product(H, W, N):
    rng = np.random.default_rng(300 + H * W + N)
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 3.0, 0.5)
    sig, _ = oracle.schedule(3.0, N)
    src = rng.normal(size=(H, W))
    x = src.ravel().copy()
    n = H * W
    for s in sig:
        r = s * np.sqrt(3.0)
        Hm = np.zeros((n, n))
        for y in range(H):
            idx = y * W + np.arange(W)
            Hm[np.ix_(idx, idx)] = box_pass_dense(dX[y], r)
        Vm = np.zeros((n, n))
        for c in range(W):
            idx = np.arange(H) * W + c
            Vm[np.ix_(idx, idx)] = box_pass_dense(dY[:, c], r)
        x = Vm @ (Hm @ x)
    np.testing.assert_allclose(oracle.box_filter_d(dX, dY, sig, src).ravel(), x, rtol=0, atol=1e-13)


def test_box_filter_uniform_guide_is_a_moving_average():
    """Unit distances (flat guide): each pass averages the samples within floor(r) positions, a
    plain moving average truncated at the borders."""
    H, W = 1, 40
    I = np.full((1, H, W), 0.5)
    src = np.random.default_rng(5).normal(size=(H, W))
    dX, dY = oracle.distances(I, 4.0, 0.2)
    sig = np.array([2.1])  # r = 3.64: windows of 3 samples on each side
    out = oracle.box_filter_d(dX, dY, sig, src)[0]
    ref = np.array([src[0, max(0, i - 3):i + 4].mean() for i in range(W)])
    np.testing.assert_allclose(out, ref, rtol=0, atol=1e-14)


def test_box_filter_constants_and_edges():
    rng = np.random.default_rng(6)
    I = rand_guide(rng, 3, 10, 12)
    out = oracle.box_filter(I, np.full((10, 12), -1.25), 6.0, 0.3)
    np.testing.assert_allclose(out, -1.25, rtol=0, atol=1e-14)
    # a strong guide edge (distance far above every radius) is never crossed
    G = np.zeros((1, 6, 10))
    G[:, :, 5:] = 1.0
    src = np.where(np.arange(10) < 5, 2.0, -3.0)[None, :].repeat(6, 0) + 0.0
    out = oracle.box_filter(G, src, 6.0, 0.001)
    np.testing.assert_allclose(out[:, :5], 2.0, atol=1e-14)
    np.testing.assert_allclose(out[:, 5:], -3.0, atol=1e-14)


def test_box_solve_one_step_and_fixed_point():
    """The solve with the box kernel: one GD step equals the dense update with the dense box
    matrix, and many Jacobi steps reach the dense solution of (lambda (I - A) + C) z = C t."""
    rng = np.random.default_rng(77)
    H, W = 4, 5
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 3.0, 0.5)
    sig, _ = oracle.schedule(3.0, 2)
    n = H * W
    A = np.eye(n)
    for s in sig:
        r = s * np.sqrt(3.0)
        Hm = np.zeros((n, n))
        for y in range(H):
            idx = y * W + np.arange(W)
            Hm[np.ix_(idx, idx)] = box_pass_dense(dX[y], r)
        Vm = np.zeros((n, n))
        for cx in range(W):
            idx = np.arange(H) * W + cx
            Vm[np.ix_(idx, idx)] = box_pass_dense(dY[:, cx], r)
        A = Vm @ Hm @ A
    t = rng.normal(size=(H, W))
    c = rng.uniform(0.2, 1.0, (H, W))
    lam, eta = 0.8, 0.99
    z1 = oracle.solve_d(dX, dY, t, c, lam=lam, sigma_s=3.0, passes=2, iterations=1, kernel=oracle.KERNEL_BOX)
    tf, cf = t.ravel(), c.ravel()
    ref = tf - eta * (lam * (tf - A @ tf) + cf * (tf - tf))
    np.testing.assert_allclose(z1.ravel(), ref, rtol=0, atol=1e-13)
    zK = oracle.solve_d(dX, dY, t, c, lam=lam, sigma_s=3.0, passes=2, iterations=3000, update=oracle.UPDATE_JACOBI,
                        kernel=oracle.KERNEL_BOX)
    zs = np.linalg.solve(lam * (np.eye(n) - A) + np.diag(cf), cf * tf)
    np.testing.assert_allclose(zK.ravel(), zs, rtol=0, atol=1e-9)


# ---------------------------------------------------------------- conjugate gradients on Eq. 2
def test_cg_reaches_the_minimiser_of_eq2():
    """After n steps (exact arithmetic) CG on the SPD system reaches the dense solution of
    (lambda (I - A)^T (I - A) + 2C) z = 2 C t; the gradient of Eq. 2 vanishes there."""
    rng = np.random.default_rng(81)
    H, W = 4, 6
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 5.0, 0.4)
    _, a = oracle.schedule(5.0, 3)
    A = dense_filter_matrix(dX, dY, a)
    t = rng.normal(size=(H, W))
    c = rng.uniform(0.1, 1.0, (H, W))
    lam = 1.3
    n = H * W
    B = np.eye(n) - A
    M = lam * B.T @ B + 2 * np.diag(c.ravel())
    zs = np.linalg.solve(M, 2 * c.ravel() * t.ravel())
    z = oracle.solve_cg_d(dX, dY, t, c, lam=lam, sigma_s=5.0, iterations=3 * n)
    np.testing.assert_allclose(z.ravel(), zs, rtol=0, atol=1e-10)
    grad = M @ z.ravel() - 2 * c.ravel() * t.ravel()
    assert np.abs(grad).max() <= 1e-9
    # CG decreases the objective monotonically along its iterates (the energy norm of the error)
    F = lambda v: 0.5 * lam * np.sum((B @ v) ** 2) + np.sum(c.ravel() * (v - t.ravel()) ** 2)
    vals = [F(oracle.solve_cg_d(dX, dY, t, c, lam=lam, sigma_s=5.0, iterations=k).ravel()) for k in range(0, 8)]
    assert all(vals[i + 1] <= vals[i] + 1e-12 for i in range(7))


def test_cg_iterates_minimise_over_the_krylov_space():
    """K steps of CG from z_init give the minimiser of 1/2 z^T M z - b^T z over z_init plus the Krylov
    space span{r0, M r0, ..., M^(K-1) r0}, r0 = b - M z_init (M = lambda (I - A)^T (I - A) + 2C, dense
    from unit vectors; b = 2Ct): pins the number of steps and the starting point, which
    convergence alone does not."""
    rng = np.random.default_rng(83)
    H, W = 4, 5
    I = rand_guide(rng, 3, H, W)
    dX, dY = oracle.distances(I, 5.0, 0.4)
    _, a = oracle.schedule(5.0, 3)
    A = dense_filter_matrix(dX, dY, a)
    t, z0 = rng.normal(size=(H, W)), rng.normal(size=(H, W))
    c = rng.uniform(0.1, 1.0, (H, W))
    lam = 0.8
    n = H * W
    B = np.eye(n) - A
    M = lam * B.T @ B + 2 * np.diag(c.ravel())
    b = 2 * c.ravel() * t.ravel()
    r0 = b - M @ z0.ravel()
    for K in (0, 1, 2, 4):
        want = z0.ravel().copy()
        if K:
            V, _ = np.linalg.qr(np.stack([np.linalg.matrix_power(M, j) @ r0 for j in range(K)], axis=1))
            want = want + V @ np.linalg.solve(V.T @ M @ V, V.T @ r0)
        got = oracle.solve_cg_d(dX, dY, t, c, lam=lam, sigma_s=5.0, iterations=K, z_init=z0).ravel()
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-9 * max(1.0, np.abs(want).max()))
        if K:
            assert np.abs(got - z0.ravel()).max() > 1e-3  # each case moves away from z_init


def test_fixed_point_keeps_pixels_without_data_or_smoothness():
    """Reading of Eq. 4 where lambda + c = 0: the fixed-point update leaves such a pixel at z_k.  With
    lambda = 0 every pixel with c > 0 takes t and every pixel with c = 0 keeps z_init, after any
    number of iterations; in reverse mode the gradient of a c = 0 pixel passes straight to z_init
    and that of a c > 0 pixel to t."""
    rng = np.random.default_rng(24)
    H, W = 6, 7
    I = rand_guide(rng, 3, H, W)
    t, z0 = rng.random((H, W)), rng.random((H, W))
    c = rng.uniform(0.2, 1.0, (H, W))
    c[rng.random((H, W)) < 0.4] = 0.0
    assert (c == 0).any() and (c > 0).any()
    kw = dict(lam=0.0, sigma_s=6.0, sigma_r=0.3, iterations=3, update=oracle.UPDATE_JACOBI)
    z = oracle.solve(I, t, c, z_init=z0, **kw)
    np.testing.assert_allclose(z, np.where(c > 0, t, z0), rtol=0, atol=1e-15)
    gz = rng.normal(size=(H, W))
    g = oracle.solve_backward(I, t, c, gz, z_init=z0, **kw)
    np.testing.assert_allclose(g["z_init"], np.where(c == 0, gz, 0.0), rtol=0, atol=1e-14)
    np.testing.assert_allclose(g["t"], np.where(c > 0, gz, 0.0), rtol=0, atol=1e-14)


def test_cg_fixed_point_differs_from_eq4():
    """The minimiser of Eq. 2 is not the fixed point of the paper's update (Eq. 4): the two agree
    only when the target already is edge-aware smooth, e.g. a constant."""
    rng = np.random.default_rng(82)
    I = rand_guide(rng, 3, 5, 5)
    t = rng.normal(size=(5, 5))
    c = rng.uniform(0.2, 1.0, (5, 5))
    zcg = oracle.solve_cg(I, t, c, lam=1.0, sigma_s=4.0, sigma_r=0.3, iterations=200)
    zj = oracle.solve(I, t, c, lam=1.0, sigma_s=4.0, sigma_r=0.3, iterations=3000, update=oracle.UPDATE_JACOBI)
    assert np.abs(zcg - zj).max() > 1e-3
    tc = np.full((5, 5), 0.4)
    np.testing.assert_allclose(oracle.solve_cg(I, tc, c, lam=1.0, sigma_s=4.0, sigma_r=0.3, iterations=30), tc,
                               atol=1e-12)


# ---------------------------------------------------------------- Charbonnier target term (§4)
def test_charbonnier_step_is_the_gradient_of_the_loss():
    """One gradient step with the Charbonnier loss c sqrt((z - t)^2 + eps^2) on the target term:
    its data part is the derivative of that loss, taken here by central differences of the loss
    itself (it is separable, so elementwise), and its smoothness part that of Eq. 3."""
    I, t, c = _small()
    rng = np.random.default_rng(5)
    z0 = t + rng.normal(0, 0.01, t.shape)  # residuals on both sides of eps = 0.001 and 0.05
    for eps in (1e-3, 0.05):
        z1 = oracle.solve(I, t, c, lam=0.9, sigma_s=8.0, sigma_r=0.2, step=0.7, iterations=1, z_init=z0,
                          charbonnier_eps=eps)
        zbar = oracle.filter(I, z0, 8.0, 0.2)
        h = 1e-4 * eps
        loss = lambda z: c * np.sqrt((z - t) ** 2 + eps ** 2)
        g = (loss(z0 + h) - loss(z0 - h)) / (2 * h)
        np.testing.assert_allclose(z1, z0 - 0.7 * (0.9 * (z0 - zbar) + g), rtol=0, atol=1e-8)


def test_charbonnier_limits():
    """eps >> |z - t|: c eps rho'(r) = c r (1 + O(r^2 / eps^2)), so the solve with confidence c eps
    is the solve of Eq. 3 with c.  eps << |z - t|: rho'(r) = sign(r), the L1 (sub)gradient step."""
    I, t, c = _small()
    kw = dict(lam=0.9, sigma_s=8.0, sigma_r=0.2, step=0.99)
    eps = 1e6
    np.testing.assert_allclose(oracle.solve(I, t, c * eps, iterations=5, charbonnier_eps=eps, **kw),
                               oracle.solve(I, t, c, iterations=5, **kw), rtol=0, atol=1e-9)
    rng = np.random.default_rng(6)
    z0 = t + rng.choice([-0.5, 0.5], t.shape)
    z1 = oracle.solve(I, t, c, iterations=1, z_init=z0, charbonnier_eps=1e-9, **kw)
    zbar = oracle.filter(I, z0, 8.0, 0.2)
    np.testing.assert_allclose(z1, z0 - 0.99 * (0.9 * (z0 - zbar) + c * np.sign(z0 - t)), rtol=0, atol=1e-12)


# ---------------------------------------------------------------- Charbonnier loss, fixed point of Eq. 4
def test_charbonnier_fixed_point_step_descends_its_pixel_objective():
    """One fixed-point step with the Charbonnier loss is a majorize-minimize step: with z_bar = A z_k
    held, every pixel's h(z) = lambda/2 (z - z_bar)^2 + c sqrt((z - t)^2 + eps^2) does not increase
    from z_k to z_{k+1} (at the paper's eps = 0.001 and at 0.05, residuals on both sides of eps)."""
    I, t, c = _small(H=9, W=11, seed=41)
    rng = np.random.default_rng(41)
    for eps in (1e-3, 0.05):
        for spread in (1e-3, 0.3):
            z0 = t + rng.normal(0, spread, t.shape)
            z1 = oracle.solve(I, t, c, lam=0.9, sigma_s=8.0, sigma_r=0.2, iterations=1, z_init=z0,
                              update=oracle.UPDATE_JACOBI, charbonnier_eps=eps)
            zbar = oracle.filter(I, z0, 8.0, 0.2)
            h = lambda z: 0.45 * (z - zbar) ** 2 + c * np.sqrt((z - t) ** 2 + eps ** 2)
            assert np.all(h(z1) <= h(z0) + 1e-12), (eps, spread, float((h(z1) - h(z0)).max()))
            # and it is a strict descent wherever z_k is not already the minimiser of h
            assert float((h(z0) - h(z1)).max()) > 0.0


@pytest.mark.parametrize("eps", [1e-3, 0.05])
def test_charbonnier_fixed_point_is_stationary_for_the_loss(eps):
    """Iterated to convergence, the fixed point satisfies the Charbonnier stationarity
    lambda (z - A z) + c rho'(z - t) = 0, rho'(r) = r / sqrt(r^2 + eps^2) -- the derivative of the loss,
    here by central differences of the loss itself -- on a dense 8 x 10 problem."""
    I, t, c = _small(H=8, W=10, seed=43)
    z = oracle.solve(I, t, c, lam=0.9, sigma_s=8.0, sigma_r=0.2, iterations=4000, update=oracle.UPDATE_JACOBI,
                     charbonnier_eps=eps)
    hh = 1e-4 * eps
    loss = lambda zz: c * np.sqrt((zz - t) ** 2 + eps ** 2)
    slope = (loss(z + hh) - loss(z - hh)) / (2 * hh)
    res = 0.9 * (z - oracle.filter(I, z, 8.0, 0.2)) + slope
    assert float(np.abs(res).max()) <= 1e-8


def test_charbonnier_fixed_point_matches_the_gradient_step_and_the_quadratic_limit():
    """Where the gradient step of the Charbonnier loss is stable (eps = 0.3, step 0.5) both readings
    converge to the same point; for eps >> |z - t| the fixed point with confidence c eps is that of
    Eq. 4 with c."""
    I, t, c = _small(H=7, W=9, seed=47)
    kw = dict(lam=0.9, sigma_s=8.0, sigma_r=0.2, iterations=3000, charbonnier_eps=0.3)
    zj = oracle.solve(I, t, c, update=oracle.UPDATE_JACOBI, **kw)
    zg = oracle.solve(I, t, c, update=oracle.UPDATE_GD, step=0.5, **kw)
    np.testing.assert_allclose(zj, zg, rtol=0, atol=1e-9)
    eps = 1e6
    np.testing.assert_allclose(
        oracle.solve(I, t, c * eps, lam=0.9, sigma_s=8.0, sigma_r=0.2, iterations=5, update=oracle.UPDATE_JACOBI,
                     charbonnier_eps=eps),
        oracle.solve(I, t, c, lam=0.9, sigma_s=8.0, sigma_r=0.2, iterations=5, update=oracle.UPDATE_JACOBI),
        rtol=0, atol=1e-9)
