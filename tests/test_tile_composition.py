"""The tiled decomposition of a solve, restated in plain Python, against the FP64 oracle (CPU).

The resident solve kernel splits every line of a pass over tiles and lanes: a row segment of a
tile is 32 lane segments, a column segment of a tile is two chunks, and every segment is reduced
to the five numbers (A, B, al, be, ga) of its causal map c_out = A c + B and its anti-causal start
k = al k_in + be c + ga.  A position then learns both carries from the segments before and after
it on its line, composed in a fixed order: lanes to the left inside the tile after the tiles to
the left, lanes to the right inside the tile before the tiles to the right; for columns, the
chunk above inside the tile after the tiles above, the chunk below before the tiles below.  This
test runs that order, with a narrow tile (32 lanes of 1 or 2 positions) so that small images
span several tiles with ragged last tiles, through K iterations of Eq. 3 and Eq. 4 with the
update applied as the last vertical pass replays, and compares with the oracle's sequential
sweeps.  It checks the decomposition, not the CUDA code, which the GPU tests compare with the
oracle directly.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1805_04590_gb300 import workloads

ID5 = (1.0, 0.0, 1.0, 0.0, 0.0)
ID2 = (1.0, 0.0)


def aff(f, s):  # f followed by s
    return (f[0] * s[0], s[0] * f[1] + s[1])


def coupled(f, s):
    return (f[0] * s[0], s[0] * f[1] + s[1], f[2] * s[2], f[2] * s[3] * f[0] + f[3],
            f[2] * (s[3] * f[1] + s[4]) + f[4])


def reduce_segment(x, w, w_next):
    """Five numbers of a segment: w[j] weights the step into position j, w_next the step out."""
    P, Q, r, be, ga = 1.0, 0.0, 1.0, 0.0, 0.0
    for j in range(len(x)):
        P *= w[j]
        Q = w[j] * (Q - x[j]) + x[j]
        wp = w[j + 1] if j + 1 < len(x) else w_next
        coef = r * (1.0 - wp)
        be += coef * P
        ga += coef * Q
        r *= wp
    return (P, Q, r, be, ga)


def replay(x, w, w_next, own, c_in, after):
    out = list(x)
    J = c_in
    for j in range(len(out)):
        J = w[j] * (J - out[j]) + out[j]
        out[j] = J
    K = after[3] * (own[0] * c_in + own[1]) + after[4]
    for j in range(len(out) - 1, -1, -1):
        wp = w[j + 1] if j + 1 < len(out) else w_next
        K = wp * (K - out[j]) + out[j]
        out[j] = K
    return out


def tiled_solve(g, t, c, *, lam, sigma_s, sigma_r, K, N, items, n_sm, update, step=0.99):
    _, H, W = g.shape
    dX, dY = oracle.distances(g, sigma_s, sigma_r, oracle.NORM_L1)
    TW = 32 * items
    ntx = -(-W // TW)
    nty = n_sm // ntx
    TH = -(-H // nty)
    nty = -(-H // TH)
    ch = (TH + 1) // 2
    z = np.zeros((nty * TH, ntx * TW))
    z[:H, :W] = t
    zk = z.copy()
    log2a = [-math.sqrt(2.0) / (sigma_s * math.sqrt(3.0) * 2.0 ** (N - i) / math.sqrt(4.0 ** N - 1.0) * math.log(2.0))
             for i in range(1, N + 1)]

    def wx(y, x, k2):
        return 2.0 ** (k2 * dX[y, x]) if 0 < x < W else 0.0

    def wy(y, x, k2):
        return 2.0 ** (k2 * dY[y, x]) if 0 < y < H and x < W else 0.0

    for _ in range(K):
        for i in range(N):
            k2 = log2a[i]
            for y in range(H):  # horizontal pass
                lanes, totals = {}, []
                for tx in range(ntx):
                    x0 = tx * TW
                    segs = []
                    for l in range(32):
                        xs = list(z[y, x0 + items * l:x0 + items * (l + 1)])
                        ws = [wx(y, x0 + items * l + j, k2) for j in range(items)]
                        segs.append((xs, ws, wx(y, x0 + items * (l + 1), k2), None))
                        segs[-1] = segs[-1][:3] + (reduce_segment(*segs[-1][:3]),)
                    tot = ID5
                    for s in reversed(segs):
                        tot = coupled(s[3], tot)
                    lanes[tx], totals = segs, totals + [tot]
                for tx in range(ntx):
                    tpre, tsuf = ID2, ID5
                    for j in range(tx):
                        tpre = aff(tpre, totals[j][:2])
                    for j in range(ntx - 1, tx, -1):
                        tsuf = coupled(totals[j], tsuf)
                    segs = lanes[tx]
                    for l, (xs, ws, wn, own) in enumerate(segs):
                        pre, suf = ID2, ID5
                        for m in range(l):
                            pre = aff(pre, segs[m][3][:2])
                        for m in range(31, l, -1):
                            suf = coupled(segs[m][3], suf)
                        pre, suf = aff(tpre, pre), coupled(suf, tsuf)
                        x0 = tx * TW + items * l
                        z[y, x0:x0 + items] = replay(xs, ws, wn, own, pre[1], suf)
            chunks, totals = {}, {}
            for ty in range(nty):  # vertical pass: reduce
                y0 = ty * TH
                rows = min(TH, H - y0)
                for x in range(ntx * TW):
                    cs = []
                    for s in range(2):
                        rb = min(s * ch, rows)
                        re = min(rb + ch, rows)
                        xs = [z[y0 + r, x] for r in range(rb, re)]
                        ws = [wy(y0 + r, x, k2) for r in range(rb, re)]
                        wn = wy(y0 + re, x, k2)
                        cs.append((rb, re, xs, ws, wn, reduce_segment(xs, ws, wn) if xs else ID5))
                    chunks[ty, x] = cs
                    totals[ty, x] = coupled(cs[0][5], cs[1][5])
            for ty in range(nty):  # vertical pass: compose and replay
                y0 = ty * TH
                for x in range(ntx * TW):
                    above, below = ID2, ID5
                    for q in range(ty):
                        above = aff(above, totals[q, x][:2])
                    for q in range(nty - 1, ty, -1):
                        below = coupled(totals[q, x], below)
                    cs = chunks[ty, x]
                    for s, (rb, re, xs, ws, wn, own) in enumerate(cs):
                        if not xs:
                            continue
                        pre = above if s == 0 else aff(above, cs[0][5][:2])
                        suf = coupled(cs[1][5], below) if s == 0 else below
                        for r, v in zip(range(rb, re), replay(xs, ws, wn, own, pre[1], suf)):
                            if i == N - 1 and x < W:
                                zo, tt, cc = zk[y0 + r, x], t[y0 + r, x], c[y0 + r, x]
                                if update == oracle.UPDATE_GD:
                                    v = zo - step * (lam * (zo - v) + cc * (zo - tt))
                                else:
                                    v = (lam * v + cc * tt) / (lam + cc)
                            z[y0 + r, x] = v
        zk = z.copy()
    return z[:H, :W]


# (H, W, positions per lane, SMs): several tiles across and down with ragged last tiles, a last
# tile row shorter than the chunk split, one-row and one-column images
@pytest.mark.parametrize("H,W,items,n_sm", [(13, 70, 1, 6), (20, 100, 2, 5), (7, 33, 1, 8), (40, 64, 2, 9),
                                            (1, 40, 1, 4), (30, 1, 1, 5)])
@pytest.mark.parametrize("update", [oracle.UPDATE_GD, oracle.UPDATE_JACOBI])
def test_tiled_composition_matches_the_sequential_sweeps(H, W, items, n_sm, update):
    p = workloads.random_problem(H, W, C=3, seed=H * W + update)
    g, t, c = (a.astype(np.float64) for a in (p.guide, p.target, p.conf))
    kw = dict(lam=0.9, sigma_s=8.0, sigma_r=0.2)
    z = tiled_solve(g, t, c, K=2, N=3, items=items, n_sm=n_sm, update=update, **kw)
    ref = oracle.solve(p.guide, p.target, p.conf, iterations=2, passes=3, update=update, **kw)
    assert np.abs(z - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())
