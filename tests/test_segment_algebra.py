"""The five-number segment algebra under random segmentations and association orders (CPU).

Every pass kernel splits a line into segments, reduces each segment to five numbers (A, B, al,
be, ga) — its causal map c_out = A c + B and its anti-causal start k = al k_in + be c + ga — and
composes them: the prefix of a segment from the causal maps of the segments before it, the
suffix from the five numbers of the segments after it.  The kernels compose in different orders
(warp shuffles, shared memory, clusters, tiles), so the composition must not depend on the
order.  This test cuts random lines at random points, composes the prefixes and suffixes along
random binary trees, replays every segment from its carries, and compares with the oracle's
sweeps: the normalised pass (causal then anti-causal) and the transposed pass that conjugate
gradients use (unnormalised causal sweep, normalised anti-causal sweep, then a factor 1 - w per
position), the latter against the oracle's adjoint of one horizontal pass; and the reverse mode
of a pass as the backward kernels form it (two causal maps and one five-number transform per
segment), for the input gradient and the distance gradient, also with the two-phase vertical
adjoint's compact chunk records and carries; and the unnormalised support sweeps of the support
weighting (a causal map and a two-number suffix per segment).
"""
import numpy as np
import pytest

import oracle

ID5 = (1.0, 0.0, 1.0, 0.0, 0.0)
ID2 = (1.0, 0.0)


def aff(f, s):
    return (f[0] * s[0], s[0] * f[1] + s[1])


def coupled(f, s):
    return (f[0] * s[0], s[0] * f[1] + s[1], f[2] * s[2], f[2] * s[3] * f[0] + f[3],
            f[2] * (s[3] * f[1] + s[4]) + f[4])


def fold(items, compose, identity, rng):
    """Composition of items in order, bracketed along a random binary tree."""
    if not items:
        return identity
    if len(items) == 1:
        return items[0]
    k = int(rng.integers(1, len(items)))
    return compose(fold(items[:k], compose, identity, rng), fold(items[k:], compose, identity, rng))


def reduce_segment(x, w, w_next, normalised):
    P, Q, r, be, ga = 1.0, 0.0, 1.0, 0.0, 0.0
    for j in range(len(x)):
        P *= w[j]
        Q = w[j] * (Q - x[j]) + x[j] if normalised else w[j] * Q + x[j]
        wp = w[j + 1] if j + 1 < len(x) else w_next
        coef = r * (1.0 - wp)
        be += coef * P
        ga += coef * Q
        r *= wp
    return (P, Q, r, be, ga)


def replay(x, w, w_next, own, c_in, after, normalised):
    out = list(x)
    J = c_in
    for j in range(len(out)):
        J = w[j] * (J - out[j]) + out[j] if normalised else w[j] * J + out[j]
        out[j] = J
    K = after[3] * (own[0] * c_in + own[1]) + after[4]
    for j in range(len(out) - 1, -1, -1):
        wp = w[j + 1] if j + 1 < len(out) else w_next
        K = wp * (K - out[j]) + out[j]
        out[j] = K if normalised else (1.0 - w[j]) * K
    return out


def segmented_pass(x, d, a, rng, normalised):
    n = len(x)
    w = [a ** d[j] if j > 0 else 0.0 for j in range(n)]
    cuts = sorted(set(int(v) for v in rng.integers(1, n, size=int(rng.integers(0, min(n, 12))))) if n > 1 else [])
    bounds = [0] + cuts + [n]
    segs = []
    for b, e in zip(bounds[:-1], bounds[1:]):
        w_next = w[e] if e < n else 0.0
        segs.append((b, e, w_next, reduce_segment(x[b:e], w[b:e], w_next, normalised)))
    out = np.empty(n)
    for s, (b, e, w_next, own) in enumerate(segs):
        pre = fold([g[3][:2] for g in segs[:s]], aff, ID2, rng)
        suf = fold([g[3] for g in segs[s + 1:]], coupled, ID5, rng)
        out[b:e] = replay(x[b:e], w[b:e], w_next, own, pre[1], suf, normalised)
    return out


@pytest.mark.parametrize("seed", range(12))
def test_normalised_pass_is_independent_of_segmentation_and_order(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 160))
    x = rng.normal(size=n)
    d = 1.0 + rng.exponential(3.0, n) * (rng.random(n) < 0.5)
    a = float(rng.uniform(0.3, 0.995))
    ref = oracle.anticausal(oracle.causal(x, d, a), d, a)
    for _ in range(4):
        got = segmented_pass(x, d, a, rng, normalised=True)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


@pytest.mark.parametrize("seed", range(8))
def test_transposed_pass_is_independent_of_segmentation_and_order(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 120))
    g = rng.normal(size=n)
    d = 1.0 + rng.exponential(3.0, n) * (rng.random(n) < 0.5)
    a = float(rng.uniform(0.3, 0.995))
    dX = d[None, :].copy()
    ref, _, _ = oracle.filter_adjoint(dX, np.ones((1, n)), np.array([a]), rng.normal(size=(1, n)), g[None, :])
    for _ in range(4):
        got = segmented_pass(g, d, a, rng, normalised=False)
        np.testing.assert_allclose(got, ref[0], rtol=0, atol=1e-13 * max(1.0, np.abs(ref).max()))


def adjoint_segmented(x, G, K, d, a, rng):
    """Reverse mode of one pass by segments: each segment reduces the causal map of J on the pass
    input x and the coupled transform of (h, gJ) on G = dL/dK; prefixes (both causal maps) and
    suffixes (the coupled transforms) are composed along random trees; each segment then replays
    with its carries and yields dL/dx and ln(a) w dL/dw, the gradient of its distances."""
    n = len(x)
    w = [a ** d[j] if j > 0 else 0.0 for j in range(n)]
    lna = np.log(a)
    cuts = sorted(set(int(v) for v in rng.integers(1, n, size=int(rng.integers(0, min(n, 12))))) if n > 1 else [])
    bounds = [0] + cuts + [n]
    segs = []
    for b, e in zip(bounds[:-1], bounds[1:]):
        w_next = w[e] if e < n else 0.0
        suf = reduce_segment(G[b:e], w[b:e], w_next, normalised=False)
        q = 0.0
        for j in range(b, e):
            q = w[j] * (q - x[j]) + x[j]
        segs.append((b, e, w_next, (suf[0], q), (suf[0], suf[1]), suf))
    gx, dd = np.empty(n), np.empty(n)
    for s, (b, e, w_next, own_jk, own_hg, own) in enumerate(segs):
        pre_jk = fold([g[3] for g in segs[:s]], aff, ID2, rng)
        pre_hg = fold([g[4] for g in segs[:s]], aff, ID2, rng)
        after = fold([g[5] for g in segs[s + 1:]], coupled, ID5, rng)
        jin, hin = pre_jk[1], pre_hg[1]
        gin = after[3] * (own_hg[0] * hin + own_hg[1]) + after[4]
        xs, Gs, Ks = list(x[b:e]), list(G[b:e]), list(K[b:e])
        Jp, hp = jin, hin
        for j in range(e - b):  # left to right: J, h and the parts of dL/dw that need J[n-1], h[n-1]
            J = w[b + j] * (Jp - xs[j]) + xs[j]
            Ks[j] = hp * (Ks[j] - Jp)
            xs[j] = Jp - xs[j]
            hp = w[b + j] * hp + Gs[j]
            Gs[j] = hp
            Jp = J
        g = gin
        for j in range(e - b - 1, -1, -1):  # right to left: gJ, then both gradients
            wp = w[b + j + 1] if j + 1 < e - b else w_next
            g = wp * (g - Gs[j]) + Gs[j]
            dd[b + j] = lna * w[b + j] * (g * xs[j] + Ks[j])
            gx[b + j] = (1.0 - w[b + j]) * g
    return gx, dd


@pytest.mark.parametrize("seed", range(8))
def test_pass_adjoint_is_independent_of_segmentation_and_order(seed):
    """The reverse mode of one horizontal pass (the backward kernels' form: J recomputed from the
    pass input by its causal map, the pass output K read back) against the oracle's adjoint of a
    one-row image with one pass, for both the input gradient and the distance gradient."""
    rng = np.random.default_rng(200 + seed)
    n = int(rng.integers(2, 120))
    x, G = rng.normal(size=n), rng.normal(size=n)
    d = 1.0 + rng.exponential(3.0, n) * (rng.random(n) < 0.5)
    a = float(rng.uniform(0.3, 0.995))
    K = oracle.row_pass(x[None, :], d[None, :], a)[0]
    gsrc, dXb, _ = oracle.filter_adjoint(d[None, :], np.ones((1, n)), np.array([a]), x[None, :], G[None, :])
    for _ in range(4):
        gx, dd = adjoint_segmented(x, G, K, d, a, rng)
        np.testing.assert_allclose(gx, gsrc[0], rtol=0, atol=1e-12 * max(1.0, np.abs(gsrc).max()))
        np.testing.assert_allclose(dd[1:], dXb[0, 1:], rtol=0, atol=1e-12 * max(1.0, np.abs(dXb).max()))


def adjoint_two_phase(x, G, K, d, a, rng):
    """The reverse mode of one pass as the two-phase vertical adjoint forms it: the line in chunks
    of segments (CTAs of warps).  Each chunk keeps six numbers: the coupled transform of its
    segments composed (A, B, al, be, ga) and the B of their composed causal map of J; the J and h
    maps share A, and the h map is the transform's (A, B).  The chunks' carries keep four: J and h
    entering from above (the B of the composed maps; their A is taken as 1) and be, ga of
    everything below.  Each segment then composes its chunk's carry with the segments of its own
    chunk and replays as in adjoint_segmented."""
    n = len(x)
    w = [a ** d[j] if j > 0 else 0.0 for j in range(n)]
    lna = np.log(a)

    def cuts(b, e, k):
        c = sorted(set(int(v) for v in rng.integers(b + 1, e, size=int(rng.integers(0, k)))) if e - b > 1 else [])
        return [b] + c + [e]

    chunks = []
    cb = cuts(0, n, min(n, 10))
    for b, e in zip(cb[:-1], cb[1:]):
        segs = []
        sb = cuts(b, e, min(e - b, 6))
        for sb0, se0 in zip(sb[:-1], sb[1:]):
            w_next = w[se0] if se0 < n else 0.0
            suf = reduce_segment(G[sb0:se0], w[sb0:se0], w_next, normalised=False)
            q = 0.0
            for j in range(sb0, se0):
                q = w[j] * (q - x[j]) + x[j]
            segs.append((sb0, se0, w_next, (suf[0], q), (suf[0], suf[1]), suf))
        tot = fold([g[5] for g in segs], coupled, ID5, rng)
        jk = fold([g[3] for g in segs], aff, ID2, rng)
        chunks.append((segs, tot + (jk[1],)))  # the six numbers of the chunk
    # carries from the records alone
    carries = []
    for c in range(len(chunks)):
        pre_jk = fold([(r[0], r[5]) for _, r in chunks[:c]], aff, ID2, rng)
        pre_hg = fold([(r[0], r[1]) for _, r in chunks[:c]], aff, ID2, rng)
        after = fold([r[:5] for _, r in chunks[c + 1:]], coupled, ID5, rng)
        carries.append((pre_jk[1], pre_hg[1], after[3], after[4]))
    gx, dd = np.empty(n), np.empty(n)
    for c, (segs, _) in enumerate(chunks):
        cj, ch, cbe, cga = carries[c]
        for s, (b, e, w_next, own_jk, own_hg, own) in enumerate(segs):
            pre_jk = fold([(1.0, cj)] + [g[3] for g in segs[:s]], aff, ID2, rng)
            pre_hg = fold([(1.0, ch)] + [g[4] for g in segs[:s]], aff, ID2, rng)
            after = fold([g[5] for g in segs[s + 1:]] + [(1.0, 0.0, 1.0, cbe, cga)], coupled, ID5, rng)
            jin, hin = pre_jk[1], pre_hg[1]
            gin = after[3] * (own_hg[0] * hin + own_hg[1]) + after[4]
            xs, Gs, Ks = list(x[b:e]), list(G[b:e]), list(K[b:e])
            Jp, hp = jin, hin
            for j in range(e - b):
                J = w[b + j] * (Jp - xs[j]) + xs[j]
                Ks[j] = hp * (Ks[j] - Jp)
                xs[j] = Jp - xs[j]
                hp = w[b + j] * hp + Gs[j]
                Gs[j] = hp
                Jp = J
            g = gin
            for j in range(e - b - 1, -1, -1):
                wp = w[b + j + 1] if j + 1 < e - b else w_next
                g = wp * (g - Gs[j]) + Gs[j]
                dd[b + j] = lna * w[b + j] * (g * xs[j] + Ks[j])
                gx[b + j] = (1.0 - w[b + j]) * g
    return gx, dd


@pytest.mark.parametrize("seed", range(8))
def test_two_phase_adjoint_records_suffice(seed):
    """The two-phase vertical adjoint's compact chunk records (six numbers) and carries (four)
    give the oracle's adjoint of a one-row pass, for any chunking, segmentation and order."""
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(2, 150))
    x, G = rng.normal(size=n), rng.normal(size=n)
    d = 1.0 + rng.exponential(3.0, n) * (rng.random(n) < 0.5)
    a = float(rng.uniform(0.3, 0.995))
    K = oracle.row_pass(x[None, :], d[None, :], a)[0]
    gsrc, dXb, _ = oracle.filter_adjoint(d[None, :], np.ones((1, n)), np.array([a]), x[None, :], G[None, :])
    for _ in range(4):
        gx, dd = adjoint_two_phase(x, G, K, d, a, rng)
        np.testing.assert_allclose(gx, gsrc[0], rtol=0, atol=1e-12 * max(1.0, np.abs(gsrc).max()))
        np.testing.assert_allclose(dd[1:], dXb[0, 1:], rtol=0, atol=1e-12 * max(1.0, np.abs(dXb).max()))


def support_segmented(x, d, a, rng):
    """Support sweeps by segments, as the support pass kernels run them: P[n] = x[n] + w_n P[n-1]
    composes as causal maps (A, B), Q[n] = x[n] + w_{n+1} Q[n+1] as pairs (al, de) with
    Q_start = al Q_in + de; each segment replays P + Q - x from its two carries."""
    n = len(x)
    w = [a ** d[j] if j > 0 else 0.0 for j in range(n)]
    cuts = sorted(set(int(v) for v in rng.integers(1, n, size=int(rng.integers(0, min(n, 12))))) if n > 1 else [])
    bounds = [0] + cuts + [n]
    segs = []
    for b, e in zip(bounds[:-1], bounds[1:]):
        A, B, r, de = 1.0, 0.0, 1.0, 0.0
        for j in range(b, e):
            A *= w[j]
            B = w[j] * B + x[j]
            de += r * x[j]
            r *= w[j + 1] if j + 1 < n else 0.0
        segs.append((b, e, (A, B), (r, de)))
    out = np.empty(n)
    for s, (b, e, _, _) in enumerate(segs):
        pre = fold([g[2] for g in segs[:s]], aff, ID2, rng)
        suf = fold([g[3] for g in segs[s + 1:]], lambda f, g: (f[0] * g[0], f[0] * g[1] + f[1]), (1.0, 0.0), rng)
        P, Pv = pre[1], []
        for j in range(b, e):
            P = w[j] * P + x[j]
            Pv.append(P)
        Q = suf[1]
        for j in range(e - 1, b - 1, -1):
            Q = (w[j + 1] if j + 1 < n else 0.0) * Q + x[j]
            out[j] = Pv[j - b] + Q - x[j]
    return out


@pytest.mark.parametrize("seed", range(6))
def test_support_sweeps_are_independent_of_segmentation_and_order(seed):
    """The support S = sum_j W_ij of the unnormalised kernel (rows on ones, columns on the row
    result) by segments in random orders, against the oracle's support."""
    rng = np.random.default_rng(300 + seed)
    H, W = int(rng.integers(2, 30)), int(rng.integers(2, 40))
    dX = 1.0 + rng.exponential(3.0, (H, W)) * (rng.random((H, W)) < 0.5)
    dY = 1.0 + rng.exponential(3.0, (H, W)) * (rng.random((H, W)) < 0.5)
    sigma_s = float(rng.uniform(2.0, 20.0))
    a = float(np.exp(-np.sqrt(2.0) / sigma_s))
    ref, _ = oracle.support(dX, dY, sigma_s)
    rows = np.stack([support_segmented(np.ones(W), dX[y], a, rng) for y in range(H)])
    got = np.stack([support_segmented(rows[:, x], dY[:, x], a, rng) for x in range(W)], axis=1)
    np.testing.assert_allclose(got, ref, rtol=1e-13, atol=0)
