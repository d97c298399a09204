"""Seeded synthetic workloads shaped like the paper's experiments.

This module only draws inputs (guides, targets, confidences) and names the
solver parameters of each workload; it holds none of the solver's arithmetic,
and both the CUDA path and the FP64 oracle consume what it returns.  Every
generator uses numpy's PCG64 with a fixed seed (1000 + workload index unless
given), so the same call returns the same arrays on any machine.

Workloads (sizes are W x H):
  0 ``plain``       256 x 256, 3-channel Voronoi guide (32 cells), per-cell depth
                    target with noise and 5% outliers, confidence U(0.2, 1).
  1 ``stereo``      2880 x 1988 RGB (the full Middlebury size), 2000 cells with
                    colour gradients, piecewise-planar disparity 0..300 px,
                    10% outliers, confidence from the residual (stands in for
                    the Middlebury stereo experiment of §4, dataset absent).
  2 ``depth_sr``    batch 8 x 2048 x 1536 RGB, 128 x 96 piecewise-smooth depth
                    bilinearly upsampled x16 as target, confidence 1 at the
                    sample sites and 0.01 elsewhere (stands in for the Ferstl
                    depth super-resolution benchmark of §4, dataset absent).
  3 ``batched``     64 images, H ~ U{240..1080}, W ~ U{320..1920}, each built
                    like workload 0.
  4 ``multispectral`` 10000 x 10000, 16 bands (smooth fields + Voronoi edges),
                    single-channel target with noise and 5% outliers,
                    confidence U(0.1, 1) (satellite-shaped imagery, §1).

Voronoi cells: workload 0 and 3 take the exact nearest of their 32 seeds
(ties to the lower index).  Larger seed counts use a jittered grid (one seed
per grid cell, uniform inside it) and take the nearest seed among the 3 x 3
neighbouring grid cells.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional

import numpy as np


@dataclasses.dataclass
class SolverParams:
    """Solver parameters of a workload (names follow the paper)."""
    lam: float
    sigma_s: float
    sigma_r: float
    iterations: int
    passes: int = 3
    step: float = 0.99


@dataclasses.dataclass
class Problem:
    """One image: guide (C, H, W), target (H, W), confidence (H, W), float32, C-contiguous."""
    guide: np.ndarray
    target: np.ndarray
    conf: np.ndarray
    truth: Optional[np.ndarray] = None

    def __post_init__(self):
        self.guide = np.ascontiguousarray(self.guide, dtype=np.float32)
        self.target = np.ascontiguousarray(self.target, dtype=np.float32)
        self.conf = np.ascontiguousarray(self.conf, dtype=np.float32)

    @property
    def shape(self):
        return self.target.shape


@dataclasses.dataclass
class Workload:
    name: str
    problems: List[Problem]
    params: SolverParams

    @property
    def megapixels(self) -> float:
        return sum(p.target.size for p in self.problems) / 1e6


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def voronoi_exact(H, W, seeds_yx):
    """Label map of the nearest seed (ties -> lower index)."""
    yy = np.arange(H, dtype=np.float64)[:, None]
    xx = np.arange(W, dtype=np.float64)[None, :]
    best = np.full((H, W), np.inf)
    lab = np.zeros((H, W), dtype=np.int32)
    for i, (sy, sx) in enumerate(seeds_yx):
        d2 = (yy - sy) ** 2 + (xx - sx) ** 2
        m = d2 < best
        best[m] = d2[m]
        lab[m] = i
    return lab


def voronoi_grid(H, W, gy, gx, rng, row_block=512):
    """Jittered-grid cells: one seed per grid cell (gy x gx grid), each pixel
    labelled by the nearest seed among the 3 x 3 neighbouring grid cells.
    Returns (labels (H, W) int32, seeds (gy*gx, 2) as (y, x))."""
    ch = H / gy
    cw = W / gx
    sy = (np.arange(gy)[:, None] + rng.random((gy, gx))) * ch
    sx = (np.arange(gx)[None, :] + rng.random((gy, gx))) * cw
    lab = np.empty((H, W), dtype=np.int32)
    xs = np.arange(W, dtype=np.float32)
    cx = np.minimum((xs / cw).astype(np.int64), gx - 1)
    for y0 in range(0, H, row_block):
        y1 = min(H, y0 + row_block)
        ys = np.arange(y0, y1, dtype=np.float32)
        cy = np.minimum((ys / ch).astype(np.int64), gy - 1)
        best = np.full((y1 - y0, W), np.inf, dtype=np.float32)
        bl = np.zeros((y1 - y0, W), dtype=np.int32)
        for dy in (-1, 0, 1):
            ny = np.clip(cy + dy, 0, gy - 1)
            for dx in (-1, 0, 1):
                nx = np.clip(cx + dx, 0, gx - 1)
                idx = ny[:, None] * gx + nx[None, :]
                py = sy.reshape(-1)[idx].astype(np.float32)
                px = sx.reshape(-1)[idx].astype(np.float32)
                d2 = (py - ys[:, None]) ** 2 + (px - xs[None, :]) ** 2
                m = d2 < best
                best[m] = d2[m]
                bl[m] = idx[m]
        lab[y0:y1] = bl
    seeds = np.stack([sy.reshape(-1), sx.reshape(-1)], axis=1)
    return lab, seeds


def plain_image(H, W, rng, cells=32, channels=3):
    """Workload-0 style image: Voronoi guide, per-cell depth target."""
    seeds = np.stack([rng.random(cells) * H, rng.random(cells) * W], axis=1)
    lab = voronoi_exact(H, W, seeds)
    colour = rng.random((cells, channels))
    guide = colour[lab].transpose(2, 0, 1) + rng.normal(0.0, 0.02, (channels, H, W))
    guide = np.clip(guide, 0.0, 1.0).astype(np.float32)
    depth = rng.random(cells)
    truth = depth[lab]
    target = truth + rng.normal(0.0, 0.05, (H, W))
    out = rng.random((H, W)) < 0.05
    target = np.where(out, rng.random((H, W)), target).astype(np.float32)
    conf = rng.uniform(0.2, 1.0, (H, W)).astype(np.float32)
    return Problem(guide, target, conf, truth.astype(np.float32))


def workload_plain(seed=1000, H=256, W=256) -> Workload:
    return Workload("plain", [plain_image(H, W, _rng(seed))],
                    SolverParams(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=10))


def _gradient_cells(H, W, rng, gy, gx):
    """Voronoi cells with per-cell colour plus a linear colour gradient and a
    per-cell disparity plane; returns (guide (3,H,W), truth (H,W), labels)."""
    lab, seeds = voronoi_grid(H, W, gy, gx, rng)
    n = gy * gx
    base = rng.random((n, 3)).astype(np.float32)
    grad = rng.uniform(-1.0, 1.0, (n, 3, 2)).astype(np.float32) * (0.15 / max(H / gy, W / gx))
    d0 = rng.uniform(20.0, 280.0, n).astype(np.float32)
    dslope = rng.uniform(-1.0, 1.0, (n, 2)).astype(np.float32) * (20.0 / max(H / gy, W / gx))
    yy = np.arange(H, dtype=np.float32)[:, None]
    xx = np.arange(W, dtype=np.float32)[None, :]
    ry = yy - seeds[lab, 0].astype(np.float32)
    rx = xx - seeds[lab, 1].astype(np.float32)
    guide = np.empty((3, H, W), dtype=np.float32)
    for c in range(3):
        guide[c] = base[lab, c] + grad[lab, c, 0] * ry + grad[lab, c, 1] * rx
    np.clip(guide, 0.0, 1.0, out=guide)
    truth = np.clip(d0[lab] + dslope[lab, 0] * ry + dslope[lab, 1] * rx, 0.0, 300.0).astype(np.float32)
    return guide, truth, lab


def stereo_image(H, W, rng, gy, gx):
    guide, truth, _ = _gradient_cells(H, W, rng, gy, gx)
    target = truth + rng.normal(0.0, 1.0, (H, W)).astype(np.float32)
    out = rng.random((H, W)) < 0.10
    target = np.where(out, rng.uniform(0.0, 300.0, (H, W)).astype(np.float32), target).astype(np.float32)
    res = np.abs(target - truth)
    conf = np.clip(1.0 - res / max(float(res.max()), 1e-12), 0.05, 1.0).astype(np.float32)
    return Problem(guide, target, conf, truth)


def workload_stereo(seed=1001, H=1988, W=2880) -> Workload:
    """2880 x 1988 RGB, 2000 cells (a 40 x 50 jittered grid at full size)."""
    gy = max(1, round(40 * H / 1988))
    gx = max(1, round(50 * W / 2880))
    return Workload("stereo", [stereo_image(H, W, _rng(seed), gy, gx)],
                    SolverParams(lam=0.99, sigma_s=16.0, sigma_r=0.1, iterations=20))


def bilinear_upsample(lr, factor):
    """Bilinear upsampling by an integer factor with half-pixel centres
    (source coordinate (i + 0.5) / factor - 0.5, clamped at the borders)."""
    h, w = lr.shape
    H, W = h * factor, w * factor

    def coords(n_out, n_in):
        s = (np.arange(n_out) + 0.5) / factor - 0.5
        s = np.clip(s, 0.0, n_in - 1)
        i0 = np.floor(s).astype(np.int64)
        i1 = np.minimum(i0 + 1, n_in - 1)
        return i0, i1, s - i0

    y0, y1, fy = coords(H, h)
    x0, x1, fx = coords(W, w)
    top = lr[y0][:, x0] * (1 - fx)[None, :] + lr[y0][:, x1] * fx[None, :]
    bot = lr[y1][:, x0] * (1 - fx)[None, :] + lr[y1][:, x1] * fx[None, :]
    return top * (1 - fy)[:, None] + bot * fy[:, None]


def depth_sr_image(H, W, rng, factor=16):
    gy = max(1, H // 48)
    gx = max(1, W // 48)
    guide, truth, _ = _gradient_cells(H, W, rng, gy, gx)
    truth = truth / 300.0
    h, w = H // factor, W // factor
    sy = np.arange(h) * factor + factor // 2
    sx = np.arange(w) * factor + factor // 2
    lr = truth[sy][:, sx].astype(np.float64)
    target = bilinear_upsample(lr, factor).astype(np.float32)
    conf = np.full((H, W), 0.01, dtype=np.float32)
    conf[np.ix_(sy, sx)] = 1.0
    return Problem(guide, target, conf, truth.astype(np.float32))


def workload_depth_sr(seed=1002, batch=8, H=1536, W=2048, factor=16) -> Workload:
    """x16 depth super-resolution; sigma_s = 20 * 2^f with f = log2(16) = 4."""
    rng = _rng(seed)
    probs = [depth_sr_image(H, W, rng, factor) for _ in range(batch)]
    f = int(round(np.log2(factor)))
    return Workload("depth_sr", probs, SolverParams(lam=0.99, sigma_s=20.0 * 2 ** f, sigma_r=0.25, iterations=10))


def workload_batched(seed=1003, n=64, hmin=240, hmax=1080, wmin=320, wmax=1920) -> Workload:
    rng = _rng(seed)
    hs = rng.integers(hmin, hmax + 1, n)
    ws = rng.integers(wmin, wmax + 1, n)
    probs = [plain_image(int(h), int(w), rng) for h, w in zip(hs, ws)]
    return Workload("batched", probs, SolverParams(lam=1.0, sigma_s=8.0, sigma_r=0.2, iterations=10))


def multispectral_image(H, W, rng, bands=16, gy=100, gx=100, sinusoids=8):
    """Bands = sum of separable low-frequency sinusoids + per-cell Voronoi
    offsets, each band scaled to [0, 1]; target = smooth + cell steps + noise."""
    lab, _ = voronoi_grid(H, W, gy, gx, rng)
    yy = np.arange(H, dtype=np.float32)
    xx = np.arange(W, dtype=np.float32)
    guide = np.empty((bands, H, W), dtype=np.float32)
    for b in range(bands):
        f = np.zeros((H, W), dtype=np.float32)
        for _ in range(sinusoids):
            ky, kx = rng.uniform(0.5, 4.0, 2) * (2 * np.pi)
            py, px = rng.uniform(0, 2 * np.pi, 2)
            amp = np.float32(rng.uniform(0.2, 1.0))
            f += amp * np.outer(np.sin(ky * yy / H + py).astype(np.float32),
                                np.sin(kx * xx / W + px).astype(np.float32))
        off = rng.uniform(-1.0, 1.0, gy * gx).astype(np.float32)
        f += off[lab]
        lo, hi = float(f.min()), float(f.max())
        guide[b] = (f - lo) / max(hi - lo, 1e-12)
    smooth = np.outer(np.sin(2 * np.pi * yy / H).astype(np.float32), np.cos(2 * np.pi * xx / W).astype(np.float32))
    steps = rng.random(gy * gx).astype(np.float32)
    truth = 0.5 * (0.3 * smooth + 0.7 * steps[lab]) + 0.25
    target = truth + rng.normal(0.0, 0.05, (H, W)).astype(np.float32)
    out = rng.random((H, W)) < 0.05
    target = np.where(out, rng.random((H, W)).astype(np.float32), target).astype(np.float32)
    conf = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    return Problem(guide, target, conf, truth.astype(np.float32))


def workload_multispectral(seed=1004, H=10000, W=10000, bands=16) -> Workload:
    g = max(1, round(100 * min(H, W) / 10000))
    return Workload("multispectral", [multispectral_image(H, W, _rng(seed), bands, g, g)],
                    SolverParams(lam=0.99, sigma_s=32.0, sigma_r=0.1, iterations=10))


def make(index: int, **kw) -> Workload:
    """Workload by index (0..4); keyword arguments shrink sizes for tests."""
    return [workload_plain, workload_stereo, workload_depth_sr, workload_batched, workload_multispectral][index](**kw)


def random_problem(H, W, C=3, seed=0, cells=6):
    """Small random problem for parity tests: Voronoi guide with noise (no
    zero colour differences), smooth-plus-steps target, confidence U(0.1, 1)."""
    rng = _rng(seed)
    cells = max(1, min(cells, H * W))
    p = plain_image(H, W, rng, cells=cells, channels=C)
    p.guide = np.clip(p.guide + rng.normal(0, 1e-3, p.guide.shape), 0, 1).astype(np.float32)
    p.conf = rng.uniform(0.1, 1.0, (H, W)).astype(np.float32)
    return p
