"""Tiny FP64 PyTorch-CPU restatement of the solver, differentiated by autograd.

Test infrastructure used to pin the oracle's hand-written reverse mode: it is
written independently of ``oracle/dts_oracle.c`` (vectorised across lines,
one Python step per position) and is only meant for images of a few dozen
pixels per side.  The forward follows the same passages: distances (§3.2,
Eq. 8-9), the recursive filter with the per-pass schedule (§2/§3.2), the
edge-aware mean (Eq. 10) and the gradient-descent / fixed-point updates
(Eq. 3 / Eq. 4).
"""
import math

import torch


def distances(I, sigma_s, sigma_r, norm=0):
    k = sigma_s / sigma_r
    dx = I[:, :, 1:] - I[:, :, :-1]
    dy = I[:, 1:, :] - I[:, :-1, :]
    if norm == 0:
        DX = 1 + k * dx.abs().sum(0)
        DY = 1 + k * dy.abs().sum(0)
    else:
        DX = torch.sqrt(1 + k * k * (dx * dx).sum(0))
        DY = torch.sqrt(1 + k * k * (dy * dy).sum(0))
    H, W = I.shape[1:]
    one_col = torch.ones(H, 1, dtype=I.dtype)
    one_row = torch.ones(1, W, dtype=I.dtype)
    return torch.cat([one_col, DX], 1), torch.cat([one_row, DY], 0)


def _lines_pass(U, D, a):
    """Causal then anti-causal sweep along dim 1 of U (lines x length)."""
    n = U.shape[1]
    w = a ** D
    cols = [U[:, 0]]
    for j in range(1, n):
        cols.append((1 - w[:, j]) * U[:, j] + w[:, j] * cols[-1])
    out = [None] * n
    out[n - 1] = cols[n - 1]
    for j in range(n - 2, -1, -1):
        out[j] = (1 - w[:, j + 1]) * cols[j] + w[:, j + 1] * out[j + 1]
    return torch.stack(out, 1)


def schedule(sigma_s, N):
    sig = [sigma_s * math.sqrt(3.0) * 2.0 ** (N - i) / math.sqrt(4.0 ** N - 1.0) for i in range(1, N + 1)]
    return [math.exp(-math.sqrt(2.0) / s) for s in sig]


def edge_mean(z, DX, DY, a_list):
    for a in a_list:
        z = _lines_pass(z, DX, a)
        z = _lines_pass(z.t(), DY.t(), a).t()
    return z


def solve(I, t, c, lam, sigma_s, sigma_r, step=0.99, iterations=3, passes=3, norm=0, update=0, z_init=None):
    DX, DY = distances(I, sigma_s, sigma_r, norm)
    a_list = schedule(sigma_s, passes)
    z = t if z_init is None else z_init
    for _ in range(iterations):
        zb = edge_mean(z, DX, DY, a_list)
        if update == 0:
            z = z - step * (lam * (z - zb) + c * (z - t))
        else:
            z = (lam * zb + c * t) / (lam + c)
    return z
