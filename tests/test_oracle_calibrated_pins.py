"""Pins of the oracle's calibrated-array path (Eq. 1 with a 3x4 camera matrix
per camera in generalized disparity space, bilinear sampling) -- CPU only.

Each pin ties the path to something outside it: the rectified oracle (already
pinned) through matrices that reduce to it exactly, the rectified oracle on
transposed frames through a vertical array, an exhaustive table sampled with
scipy's ``map_coordinates``, and the ground truth of a noise-free plane scene
rendered through the inverse plane homographies.
"""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2003_11076_gb300 import scenes


def _rectified_matrices(b):
    cams = np.zeros((len(b), 3, 4), np.float32)
    for k, bk in enumerate(b):
        cams[k, :, :3] = np.eye(3)
        cams[k, 0, 3] = -bk
    return cams


def test_rectified_matrices_reproduce_the_rectified_oracle_exactly():
    """[I | (-b_k, 0, 0)] makes the general sampling reduce to u - d b_k on row
    v with a zero vertical weight: every output and diagnostic is identical."""
    s = scenes.small_gray(0)
    ref = O.run_scene(s)
    gen = O.run(s.images, s.seg_prior, s.baselines, s.points, s.d_min, s.d_max, s.D, s.iters,
                cameras=_rectified_matrices(s.baselines))
    for k in ("d_idx", "d", "labels", "post", "refocus", "m_margin", "e_margin", "J_t", "init_margin"):
        assert np.array_equal(gen[k], ref[k]), k


def test_vertical_array_equals_rectified_on_transposed_frame():
    """A vertical array [I | (0, -b_k, 0)] on the transposed frame samples
    columns exactly as the rectified array samples rows (the descriptor
    channels Sobel-x / Sobel-y trade places, which the variance ignores)."""
    s = scenes.small_gray(1, H=40, W=56)
    ref = O.run_scene(s)
    cams = np.zeros((s.K, 3, 4), np.float32)
    for k, bk in enumerate(s.baselines):
        cams[k, :, :3] = np.eye(3)
        cams[k, 1, 3] = -bk
    imgT = np.ascontiguousarray(s.images.transpose(0, 2, 1))
    segT = np.ascontiguousarray(s.seg_prior.transpose(0, 2, 1))
    ptsT = np.ascontiguousarray(s.points[:, [1, 0, 2]])
    gen = O.run(imgT, segT, s.baselines, ptsT, s.d_min, s.d_max, s.D, s.iters, cameras=cams)
    ok = ~O.excused(ref, tau_rel=1e-9, tau_init=1e-9) & ~O.excused(
        {k: (v.transpose(0, 2, 1) if v.ndim == 3 else v.T) for k, v in gen.items()
         if k in ("m_margin", "e_margin", "J_t", "init_margin")}, tau_rel=1e-9, tau_init=1e-9)
    assert ok.mean() > 0.95
    assert np.array_equal(gen["d_idx"].T[ok], ref["d_idx"][ok])
    assert np.array_equal(gen["labels"].T[ok], ref["labels"][ok])
    assert np.allclose(gen["post"].transpose(0, 2, 1)[:, ok], ref["post"][:, ok], atol=1e-9)
    assert np.allclose(gen["refocus"].T[ok], ref["refocus"][ok], atol=1e-12)


def _tiny_calibrated(K, H, W, seed):
    rng = np.random.default_rng(seed)
    imgs = rng.random((K, H, W)).astype(np.float32)
    seg = rng.uniform(0.02, 0.98, size=(K, H, W)).astype(np.float32)
    b = np.concatenate([[0.0], rng.uniform(-0.6, 0.6, size=K - 1)]).astype(np.float32)
    cams = scenes.calibrated_cameras(rng, b, H, W, rot_deg=4.0, shift_y=0.3, shift_z=0.1, focal_jitter=0.05)
    pts = np.stack([rng.uniform(-1, W, 6), rng.uniform(-1, H, 6), rng.uniform(0, 4, 6)], 1).astype(np.float32)
    return imgs, seg, b, cams, pts


@pytest.mark.parametrize("seed,K,H,W,D", [(1, 3, 5, 6, 5), (2, 4, 4, 5, 6), (3, 2, 6, 5, 4), (4, 1, 4, 6, 3)])
def test_calibrated_em_matches_exhaustive_table(seed, K, H, W, D):
    """Every arg-max, posterior and refocused value of the calibrated path
    agrees with the exhaustive J[d, S] table whose rays are sampled by
    scipy.ndimage.map_coordinates at the dehomogenised camera positions."""
    imgs, seg, b, cams, pts = _tiny_calibrated(K, H, W, seed)
    p = O.Params(beta=30.0)
    iters = 3
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, D, iters, params=p, cameras=cams)
    bf = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, D, iters, p, cameras=cams)
    ok = ~O.excused(out, tau_rel=1e-9, tau_init=1e-9)
    assert ok.sum() >= 6
    assert np.array_equal(out["d_idx"][ok], bf["d_idx"][ok])
    assert np.array_equal(out["labels"][ok].astype(np.int64), bf["labels"][ok])
    assert np.allclose(out["post"][:, ok], bf["post"][:, ok], atol=1e-10)
    assert np.allclose(out["refocus"][ok], bf["refocus"][ok], atol=1e-12)
    assert np.allclose(out["J_t"][-1][ok], bf["J_final"][ok], atol=1e-9)


def test_calibrated_pin_catches_planted_axis_swap(monkeypatch):
    """The table pin is sensitive to the geometry: sampling at (y, x) instead
    of (x, y) changes the result somewhere."""
    imgs, seg, b, cams, pts = _tiny_calibrated(3, 5, 6, 1)
    p = O.Params(beta=30.0)
    out = O.run(imgs, seg, b, pts, 0.0, 4.0, 5, 3, params=p, cameras=cams)
    good = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 3, p, cameras=cams)
    assert np.allclose(good["J_final"], out["J_t"][-1], atol=1e-9)
    orig = BF._position
    monkeypatch.setattr(BF, "_position", lambda cam, u, v, d: orig(cam, u, v, d)[::-1])
    bad = BF.run(imgs, seg, b, out["mu"], out["inside"], 0.0, 4.0, 5, 3, p, cameras=cams)
    assert not np.allclose(bad["J_final"], out["J_t"][-1], atol=1e-9)


def test_calibrated_plane_scene_recovers_ground_truth():
    """Noise-free, occluder-free planes seen by a non-rectified array
    (rotations up to 1.5 degrees, vertical and forward offsets, focal
    jitter): the disparity is within one level of the ground truth and every
    ray static on the interior away from plane boundaries."""
    b = [-0.2, -0.1, 0.0, 0.1, 0.2]
    H, W = 48, 80
    cams = scenes.calibrated_cameras(np.random.default_rng(77), b, H, W, rot_deg=1.5)
    s = scenes.plane_scene(13, H=H, W=W, baselines=b, planes=(4.0, 9.0), D=32, M=0, cameras=cams)
    assert s.cameras is not None and s.name.endswith("_calibrated")
    out = O.run_scene(s)
    mask = np.zeros((H, W), bool)
    mask[4:-4, 8:W - 8] = True
    u = np.arange(W)
    for ub in (0.0, 0.35 * W):
        mask[:, np.abs(u - ub) <= 5] = False
    err = np.abs(out["d"] - s.gt_disparity)[mask]
    assert np.mean(err <= 1.0) >= 0.97
    assert np.mean(out["labels"][mask] == 0b11111) >= 0.97
    # the cameras really are not rectified: the rectified model of the same
    # images misses the ground truth on most pixels
    wrong = O.run(s.images, s.seg_prior, s.baselines, s.points, s.d_min, s.d_max, s.D, s.iters)
    assert np.mean(np.abs(wrong["d"] - s.gt_disparity)[mask] <= 1.0) < 0.5
