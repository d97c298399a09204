"""The seeded synthetic workloads follow the stated input recipe (CPU, reduced sizes).

They stand in for the paper's data (Middlebury-shaped stereo, Ferstl-shaped depth
super-resolution, many uneven images, 16-band satellite-shaped imagery), none of which is
available; these checks hold each generator to the recipe the benchmark and the parity tests
rely on.
"""
import numpy as np

from paper_1805_04590_gb300 import workloads


def test_stereo_recipe():
    wl = workloads.make(1, H=199, W=288)
    p = wl.problems[0]
    assert p.guide.shape == (3, 199, 288) and p.target.shape == (199, 288)
    assert 0.0 <= p.guide.min() and p.guide.max() <= 1.0
    assert 0.0 <= p.truth.min() and p.truth.max() <= 300.0
    res = np.abs(p.target - p.truth)
    # N(0, 1) noise everywhere, 10 % of the pixels replaced by U(0, 300) outliers
    outliers = res > 5.0
    assert 0.07 < outliers.mean() < 0.12
    assert np.abs(res[~outliers]).std() < 1.2
    np.testing.assert_allclose(p.conf, np.clip(1.0 - res / res.max(), 0.05, 1.0), rtol=0, atol=1e-6)
    q = wl.params
    assert (q.lam, q.sigma_s, q.sigma_r, q.iterations, q.passes) == (0.99, 16.0, 0.1, 20, 3)


def test_depth_sr_recipe():
    wl = workloads.make(2, batch=2, H=192, W=256)
    assert len(wl.problems) == 2
    for p in wl.problems:
        sites = np.zeros(p.target.shape, dtype=bool)
        sites[8::16, 8::16] = True
        assert (p.conf[sites] == 1.0).all() and (p.conf[~sites] == np.float32(0.01)).all()
        assert p.target.min() >= p.truth.min() - 1e-6 and p.target.max() <= p.truth.max() + 1e-6
    q = wl.params
    assert q.sigma_s == 320.0 and q.sigma_r == 0.25 and q.iterations == 10  # sigma = 20 * 2^f, f = log2(16)


def test_bilinear_upsampling_reproduces_linear_ramps():
    lr = np.add.outer(np.arange(6.0) * 2.0, np.arange(5.0) * -3.0)
    up = workloads.bilinear_upsample(lr, 4)
    assert up.shape == (24, 20)
    # half-pixel centres: HR pixel i sits at LR coordinate (i + 0.5) / 4 - 0.5, clamped at the borders
    yy = np.clip((np.arange(24) + 0.5) / 4 - 0.5, 0, 5)
    xx = np.clip((np.arange(20) + 0.5) / 4 - 0.5, 0, 4)
    np.testing.assert_allclose(up, np.add.outer(yy * 2.0, xx * -3.0), rtol=0, atol=1e-12)
    np.testing.assert_array_equal(workloads.bilinear_upsample(lr, 1), lr)


def test_batched_recipe():
    wl = workloads.make(3, n=5, hmin=20, hmax=40, wmin=30, wmax=50)
    assert len(wl.problems) == 5
    for p in wl.problems:
        H, W = p.target.shape
        assert 20 <= H <= 40 and 30 <= W <= 50 and p.guide.shape == (3, H, W)
    assert len({p.target.shape for p in wl.problems}) > 1


def test_multispectral_recipe():
    wl = workloads.make(4, H=160, W=200, bands=4)
    p = wl.problems[0]
    assert p.guide.shape == (4, 160, 200)
    for b in range(4):  # every band scaled to exactly [0, 1]
        assert p.guide[b].min() == 0.0 and abs(p.guide[b].max() - 1.0) < 1e-6
    assert 0.1 <= p.conf.min() and p.conf.max() <= 1.0
    # N(0, 0.05) noise, 5 % of the pixels replaced by U(0, 1): the share of pixels more than 0.2
    # from the truth is 5 % times the chance that a uniform value falls that far from it
    far = np.abs(p.target - p.truth) > 0.2
    t = p.truth.astype(np.float64)
    expected = 0.05 * np.mean(1.0 - (np.minimum(t + 0.2, 1.0) - np.maximum(t - 0.2, 0.0)))
    assert abs(far.mean() - expected) < 5 * np.sqrt(expected / far.size)
    q = wl.params
    assert (q.lam, q.sigma_s, q.sigma_r, q.iterations) == (0.99, 32.0, 0.1, 10)
