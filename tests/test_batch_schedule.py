"""The job queue of the persistent batched solve, restated in plain Python (CPU).

The batched kernel cuts every image's solve into stages -- distances, 2 N K passes alternating
horizontal and vertical, the last update -- and every stage into jobs (groups of rows, 8-column
strips, row tiles), queued round by round (round r = stage r of every image) and taken by ticket.
Restated here from the same rules: every ticket decodes to one job and every job to one ticket;
a job's stage waits only on jobs of its image's previous stage, all with smaller tickets (so the
queue always advances); every job's rows and columns stay inside its image and within the CTA's
512 threads; together the jobs of a stage cover their image exactly once.
"""
import numpy as np
import pytest

from paper_1805_04590_gb300 import workloads

THREADS, ROW_ITEMS, JOB_PIXELS, STRIP_COLS = 512, 16, 16384, 8
MAX_ROWS, MAX_COLS = 4 * 16 * 17, 16 * 512


def shapes(H, W):
    tpr = ((W + ROW_ITEMS - 1) // ROW_ITEMS + 31) // 32 * 32
    rpb = THREADS // tpr
    gpj = max(1, JOB_PIXELS // (rpb * W))
    col_items = 9 if H <= 4 * (THREADS // 32) * 9 else 17
    spj = max(1, JOB_PIXELS // (STRIP_COLS * H))
    tile_rows = max(1, JOB_PIXELS // W)
    groups, strips = -(-H // rpb), -(-W // STRIP_COLS)
    return dict(tpr=tpr, rpb=rpb, gpj=gpj, col_items=col_items, spj=spj, tile_rows=tile_rows,
                groups=groups, strips=strips, row_jobs=-(-groups // gpj), col_jobs=-(-strips // spj),
                tile_jobs=-(-H // tile_rows))


def image_of(pre, j):
    lo, hi = 0, len(pre) - 2
    while lo < hi:
        mid = (lo + hi + 1) >> 1
        if pre[mid] <= j:
            lo = mid
        else:
            hi = mid - 1
    return lo


def decode(t, pre_tile, pre_row, pre_col, N, K, S):
    rt, rr, rc = pre_tile[-1], pre_row[-1], pre_col[-1]
    if t < rt:
        m = image_of(pre_tile, t)
        return m, 0, t - pre_tile[m]
    t -= rt
    pair = t // (rr + rc)
    if pair < N * K:
        rem = t - pair * (rr + rc)
        if rem < rr:
            m = image_of(pre_row, rem)
            return m, 1 + 2 * pair, rem - pre_row[m]
        m = image_of(pre_col, rem - rr)
        return m, 2 + 2 * pair, rem - rr - pre_col[m]
    t -= N * K * (rr + rc)
    m = image_of(pre_tile, t)
    return m, S - 1, t - pre_tile[m]


def stage_jobs(sh, s, S):
    if s in (0, S - 1):
        return sh["tile_jobs"]
    return sh["row_jobs"] if s % 2 else sh["col_jobs"]


def check_batch(sizes, N, K):
    S = 2 * N * K + 2
    sh = [shapes(H, W) for H, W in sizes]
    pre_tile, pre_row, pre_col = [0], [0], [0]
    for x in sh:
        pre_tile.append(pre_tile[-1] + x["tile_jobs"])
        pre_row.append(pre_row[-1] + x["row_jobs"])
        pre_col.append(pre_col[-1] + x["col_jobs"])
    total = 2 * pre_tile[-1] + N * K * (pre_row[-1] + pre_col[-1])
    ticket = {}
    for t in range(total):
        m, s, j = decode(t, pre_tile, pre_row, pre_col, N, K, S)
        assert 0 <= m < len(sizes) and 0 <= s < S and 0 <= j < stage_jobs(sh[m], s, S), (t, m, s, j)
        assert (m, s, j) not in ticket
        ticket[(m, s, j)] = t
    assert len(ticket) == sum(stage_jobs(x, s, S) for x in sh for s in range(S))
    # waits go to smaller tickets only
    for (m, s, j), t in ticket.items():
        if s > 0:
            assert max(ticket[(m, s - 1, q)] for q in range(stage_jobs(sh[m], s - 1, S))) < t
    # every job inside its image and its CTA; each stage covers its image exactly once
    for (H, W), x in zip(sizes, sh):
        assert x["tpr"] % 32 == 0 and x["tpr"] <= THREADS and x["rpb"] >= 1 and x["tpr"] * x["rpb"] <= THREADS
        assert x["tpr"] * ROW_ITEMS >= W  # one row group's threads hold every position of a row
        assert 4 * (THREADS // 32) * x["col_items"] >= H  # a strip job's segments hold the whole column
        rows = np.zeros(H, int)
        for j in range(x["row_jobs"]):  # a job runs row groups [j gpj, min((j + 1) gpj, groups))
            for g in range(j * x["gpj"], min((j + 1) * x["gpj"], x["groups"])):
                r = np.arange(g * x["rpb"], (g + 1) * x["rpb"])
                rows[r[r < H]] += 1
        assert (rows == 1).all()
        cols = np.zeros(W, int)
        for j in range(x["col_jobs"]):  # strips [j spj, min((j + 1) spj, strips))
            for st in range(j * x["spj"], min((j + 1) * x["spj"], x["strips"])):
                c = np.arange(st * STRIP_COLS, (st + 1) * STRIP_COLS)
                cols[c[c < W]] += 1
        assert (cols == 1).all()
        tiles = np.zeros(H, int)
        for j in range(x["tile_jobs"]):
            r = np.arange(j * x["tile_rows"], (j + 1) * x["tile_rows"])
            tiles[r[r < H]] += 1
        assert (tiles == 1).all()
    return total


def test_schedule_of_the_64_image_workload():
    """The batched workload's 64 images (240..1080 x 320..1920), K = 10, N = 3."""
    wl = workloads.make(3)
    sizes = [p.target.shape for p in wl.problems]
    assert all(H <= MAX_ROWS and W <= MAX_COLS for H, W in sizes)
    check_batch(sizes, N=3, K=10)


@pytest.mark.parametrize("sizes,N,K", [([(1, 1)], 1, 1), ([(1, 8192), (1088, 1), (577, 576)], 2, 3),
                                       ([(17, 33), (576, 9), (31, 1000), (1088, 8192)], 3, 2),
                                       ([(5, 7)] * 96, 1, 1)])
def test_schedule_at_the_edges(sizes, N, K):
    """One pixel; the widest row and the tallest column a job holds; both strip heights (9 and 17
    rows per thread, switching above 576); the most images one launch takes."""
    check_batch(sizes, N, K)
