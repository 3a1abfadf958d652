"""Pins of the support-point oracle (Sec. III-C "Disparity Prior") -- CPU only.

The oracle (support_oracle.c) is tied to an array restatement of the same
reading (scipy Sobel, padded descriptor windows, whole cost tables), to exact
matches on a noise-free integer-shift plane, to the segmentation filters, to
the uniqueness test on a periodic texture, and to occluded background
recovered from the other views.
"""
import numpy as np
import pytest

from oracle import bruteforce as BF
from oracle import oracle as O
from paper_2003_11076_gb300 import scenes


def _same(a, b):
    assert np.array_equal(a["cell_j"], b["cell_j"])
    assert np.array_equal(a["cell_src"], b["cell_src"])
    assert np.allclose(a["cell_u"], b["cell_u"], atol=1e-12)
    assert np.array_equal(a["cell_v"], b["cell_v"])


@pytest.mark.parametrize("make", [
    lambda: scenes.small_gray(0),
    lambda: scenes.small_gray(3, baselines=[-0.3, -0.1, 0.0, 0.2], D=24),
    lambda: scenes.street_rgb(2, H=60, W=96, D=32, M=20),
    lambda: scenes.random_frame(4, scale=0.1),
])
def test_support_points_match_array_restatement(make):
    s = make()
    sp = O.SupportParams(grid=4, texture=60, window=2, min_support=1)
    a = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, sp)
    b = BF.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, sp)
    assert (a["cell_j"] >= 0).sum() >= 10
    _same(a, b)


def test_support_points_restatement_catches_planted_ratio_flip(monkeypatch):
    s = scenes.small_gray(0)
    sp = O.SupportParams(grid=4, texture=60, window=2, min_support=1)
    a = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, sp)
    loose = O.SupportParams(grid=4, texture=60, window=2, min_support=1, ratio_pct=99)
    b = BF.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, loose)
    assert not np.array_equal(a["cell_j"], b["cell_j"])


def test_noise_free_integer_shift_plane_gives_exact_disparities():
    """Baselines 0, +-0.25, +-0.5 and a plane at d = 8: every target pixel is
    an exact integer shift (no other candidate rounds to the same shifts), the
    true candidate has cost 0, and every accepted point whose true targets and
    their windows stay inside the image carries d = 8."""
    b = [-0.5, -0.25, 0.0, 0.25, 0.5]
    s = scenes.plane_scene(21, H=40, W=80, baselines=b, planes=(8.0,), D=17, d_max=16.0, M=0,
                           texture_cells=(3.0, 1.5, 1.0), p_static=0.0)
    r = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D,
                         O.SupportParams(grid=4, texture=30))
    m = r["cell_j"] >= 0
    assert m.mean() > 0.5
    inner = m & (r["cell_u"] >= 5) & (r["cell_u"] <= s.W - 6)
    assert inner.sum() > 0.8 * m.sum()
    assert np.all(r["cell_j"][inner] == 8)
    assert np.all(r["cell_src"][m] == s.ref)


def test_periodic_texture_is_rejected_as_ambiguous():
    """Vertical stripes with a period shorter than the searched shift range
    match equally well one period apart: the uniqueness test rejects them."""
    K, H, W = 3, 24, 64
    b = np.array([-0.5, 0.0, 0.5], np.float32)
    u = np.arange(W)
    row = np.where((u // 2) % 2 == 0, 0.9, 0.1).astype(np.float32)  # period 4 px
    imgs = np.repeat(np.repeat(row[None, None, :], H, 1), K, 0)
    seg = np.full((K, H, W), 0.05, np.float32)
    r = O.support_points(imgs, seg, b, 0.0, 20.0, 21, O.SupportParams(grid=4, texture=10, min_support=0))
    # cells whose grid pixel keeps every candidate's targets inside the image
    # (shifts up to 10 px)
    ugrid = 4 * np.arange(r["cell_j"].shape[1]) + 2
    inner = np.broadcast_to((ugrid >= 12) & (ugrid <= W - 13), r["cell_j"].shape)
    assert ((r["cell_j"] >= 0) & inner).sum() == 0
    # the same stripes with a period longer than the shift range are matched
    row = np.where((u // 16) % 2 == 0, 0.9, 0.1).astype(np.float32)
    imgs = np.repeat(np.repeat(row[None, None, :], H, 1), K, 0)
    r = O.support_points(imgs, seg, b, 0.0, 20.0, 21, O.SupportParams(grid=4, texture=10, min_support=0))
    assert ((r["cell_j"] >= 0) & inner).sum() > 0


def test_segmentation_filters():
    """Reference points never touch a dynamic pixel of their window; points
    from the other views land on dynamic reference pixels only."""
    s = scenes.street_rgb(1, H=120, W=192, D=64, M=20)
    r = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, O.SupportParams())
    thr = np.float32(0.7)
    Pref = s.seg_prior[s.ref]
    for cj, ci in np.argwhere(r["cell_j"] >= 0):
        u, v = r["cell_u"][cj, ci], int(r["cell_v"][cj, ci])
        if r["cell_src"][cj, ci] == s.ref:
            win = Pref[max(v - 1, 0):v + 2, max(int(u) - 1, 0):int(u) + 2]
            assert np.all(win < thr)
        else:
            assert Pref[v, int(np.floor(u + 0.5))] >= thr


def test_occluded_background_is_recovered_from_other_views():
    """An occluder drawn only in the reference view hides background that
    every other camera sees: the other views supply points there, with the
    background's disparity."""
    b = [-0.2, -0.1, 0.0, 0.1, 0.2]
    s = scenes.small_gray(9, H=48, W=96, baselines=b, D=32, occluder_disparity=20.0, noise=0.0)
    # redraw: occluder only in the reference view
    rng = np.random.default_rng(5)
    from paper_2003_11076_gb300.scenes import Surface, value_noise, pixel_noise, render_scene
    ext = (-80.0, -4.0, 176.0, 52.0)
    far = Surface(6.0, None, [value_noise(rng, (6.0, 3.0, 1.5), (0.5, 0.3, 0.2), ext)])
    occ = Surface(20.0, (36, 10, 60, 38), [pixel_noise(rng, (30, 5, 66, 42))], dynamic=True, views=[2])
    imgs, dyn, _, st_disp = render_scene([far, occ], np.array(b, np.float32), 48, 96, 1)
    imgs = imgs[..., 0].astype(np.float32)
    seg = np.where(dyn, 0.9, 0.05).astype(np.float32)
    r = O.support_points(imgs, seg, np.array(b, np.float32), 0.0, 31.0, 32, O.SupportParams(grid=4, texture=40))
    other = (r["cell_j"] >= 0) & (r["cell_src"] != 2)
    assert other.sum() >= 5
    assert np.all(np.abs(np.array(r["cell_j"][other], float) - 6.0) <= 1.0)
    for cj, ci in np.argwhere(other):
        assert dyn[2, int(r["cell_v"][cj, ci]), int(np.floor(r["cell_u"][cj, ci] + 0.5))]
