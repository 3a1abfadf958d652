"""The seeded synthetic inputs follow the recipes the benchmarks and parity
tests are stated on (CPU only): shapes, camera layouts, candidate ranges,
occluder coverage, segmentation-prior distributions and support points."""
import numpy as np
import pytest

from paper_2003_11076_gb300 import scenes


def test_small_gray_recipe():
    s = scenes.small_gray(0)
    assert s.images.shape == (5, 48, 64) and s.images.dtype == np.float32
    assert s.images.min() >= 0.0 and s.images.max() <= 1.0
    assert np.allclose(np.sort(s.baselines), [-0.2, -0.1, 0.0, 0.1, 0.2]) and np.sum(s.baselines == 0) == 1
    assert (s.D, s.d_min, s.d_max, s.iters) == (32, 0.0, 31.0, 5)
    assert s.points.shape == (40, 3)
    # the occluder is drawn in the three central views only
    outer = np.abs(s.baselines) > 0.15
    assert not s.dynamic_mask[outer].any() and s.dynamic_mask[~outer].any(axis=(1, 2)).all()
    # P(dynamic) = 0.9 on occluder pixels and 0.05 elsewhere, +- 0.03
    P = s.seg_prior
    assert np.all(np.abs(P[s.dynamic_mask] - 0.9) <= 0.03 + 1e-6)
    assert np.all(np.abs(P[~s.dynamic_mask] - 0.05) <= 0.03 + 1e-6)
    # support points lie on the static background: d = ground truth + N(0, 0.3^2)
    u = np.clip(np.rint(s.points[:, 0]).astype(int), 0, 63)
    v = np.clip(np.rint(s.points[:, 1]).astype(int), 0, 47)
    err = s.points[:, 2] - s.gt_disparity[v, u]
    assert np.median(np.abs(err)) < 0.6


@pytest.mark.parametrize("frame", [0, 1])
def test_street_rgb_recipe(frame):
    s = scenes.street_rgb(frame)
    assert s.images.shape == (5, 600, 960, 3) and s.images.dtype == np.uint8
    assert np.allclose(np.sort(s.baselines), [-0.2, -0.1, 0.0, 0.1, 0.2])
    assert (s.D, s.d_min, s.d_max, s.iters) == (64, 0.0, 63.0, 10)
    assert s.points.shape == (300, 3)
    ref = int(np.flatnonzero(s.baselines == 0)[0])
    cover = s.dynamic_mask[ref].mean()
    assert 0.10 <= cover <= 0.35
    # P ~ Beta(8, 2) on person pixels (mean 0.8) and Beta(1, 15) elsewhere (mean 1/16)
    P = s.seg_prior
    assert abs(P[s.dynamic_mask].mean() - 0.8) < 0.01
    assert abs(P[~s.dynamic_mask].mean() - 1.0 / 16.0) < 0.005
    # the deterministic seed gives the same frame again
    t = scenes.street_rgb(frame)
    assert np.array_equal(s.images, t.images) and np.array_equal(s.seg_prior, t.seg_prior)
    assert np.array_equal(s.points, t.points)


def test_random_frames_recipe():
    seen_K, seen_D = set(), set()
    for i in range(24):
        # scale shrinks the rendered frame only: the seeded draws of size, K,
        # D and spacings come in the same order
        s = scenes.random_frame(i, scale=0.125)
        K, H, W = s.images.shape[:3]
        assert 40 <= W <= 160 and 30 <= H <= 128
        assert K in (3, 5, 7, 9) and s.D in (32, 64, 128)
        b = np.sort(s.baselines)
        assert np.sum(s.baselines == 0) == 1 and s.baselines[K // 2] == 0
        gaps = np.diff(b)
        assert np.all(gaps >= 0.05 - 1e-6) and np.all(gaps <= 0.25 + 1e-6)
        seen_K.add(K)
        seen_D.add(s.D)
    assert seen_K == {3, 5, 7, 9} and seen_D == {32, 64, 128}
