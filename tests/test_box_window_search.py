"""The box kernel's window search, restated in plain Python, against brute force (CPU).

Along a line the box kernel of Eq. 10 averages the positions m with |ct_m - ct_n| <= r, ct the
domain coordinate.  The kernel keeps ct as an exact integer count of 2^-23 units (FP32 distances
of at least 1 are whole multiples of 2^-23) and compares differences with R = floor(r 2^23).
Because every distance is at least 1, no window reaches more than floor(r) positions from its
centre, so each end is found by binary lifting over that range with the same number of steps,
ceil(log2(floor(r) + 1)), at every position.  This test runs that search on random lines (flat,
sparse edges, dense edges; radii from 0 to wider than the line) and compares both ends with the
windows found by testing every position.  It checks the search, not the CUDA code, which the GPU
tests compare with the oracle directly.
"""
import math

import numpy as np
import pytest

UNIT = 1 << 23


def window_ends(ct, R, rmax):
    """(lo, up) per position by binary lifting with a fixed step count (largest power of two
    <= rmax first), indexes clamped into the candidate range."""
    L = len(ct)
    top = 0
    if rmax > 0:
        top = 1
        while 2 * top <= rmax:
            top *= 2
    los, ups = [], []
    for i in range(L):
        ci = int(ct[i])
        lo, up, hb = max(0, i - rmax), i, min(L - 1, i + rmax)
        st = top
        while st > 0:
            ml = min(lo + st - 1, i)
            if ci - int(ct[ml]) > R:
                lo = ml + 1
            mu = min(up + st, hb)
            if int(ct[mu]) - ci <= R:
                up = mu
            st >>= 1
        los.append(lo)
        ups.append(up)
    return np.array(los), np.array(ups)


@pytest.mark.parametrize("L", [1, 2, 3, 31, 100, 517])
@pytest.mark.parametrize("kind", ["flat", "sparse_edges", "dense_edges"])
@pytest.mark.parametrize("r", [0.0, 0.5, 1.0, 2.0, 6.05, 24.2, 484.0, 1e5])
def test_window_ends_match_brute_force(L, kind, r):
    rng = np.random.default_rng(L * 31 + len(kind) + int(r))
    if kind == "flat":
        d = np.ones(L)
    elif kind == "sparse_edges":
        d = 1.0 + (rng.random(L) < 0.05) * 200.0
    else:
        d = 1.0 + rng.random(L) * 40.0
    d = d.astype(np.float32).astype(np.float64)
    units = np.round(d * UNIT).astype(np.int64)  # FP32 values >= 1: exact multiples of 2^-23
    units[0] = 0
    ct = np.cumsum(units)
    R = math.floor(r * UNIT)
    rmax = min(math.floor(r), L)
    lo, up = window_ends(ct, R, rmax)
    inside = np.abs(ct[None, :] - ct[:, None]) <= R
    first = inside.argmax(axis=1)
    last = L - 1 - inside[:, ::-1].argmax(axis=1)
    np.testing.assert_array_equal(lo, first)
    np.testing.assert_array_equal(up, last)
    # the windows are contiguous, so the two ends describe them fully
    assert (inside.sum(axis=1) == last - first + 1).all()
