"""Support points detected on the device (lf_set_inputs with
M = LF_DETECT_SUPPORT) against the oracle's support points: every decision is
integer or double arithmetic, so the point sets must be identical."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_11076_gb300 import scenes
from test_gpu_parity import check_parity, params_pair

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_11076_gb300 import build
    build.build()
    O.build()


def _oracle_params(sp, thr=0.7):
    return O.SupportParams(grid=sp.grid, ratio_pct=sp.ratio_pct, texture=sp.texture, window=sp.window,
                           delta=float(np.float32(sp.delta)), min_support=sp.min_support,
                           seg_threshold=float(np.float32(thr)))


def _detect(s, sp=None, device=False):
    import torch
    from paper_2003_11076_gb300 import lf
    with lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D) as ctx:
        if sp is not None:
            ctx.set_support_params(sp)
        if device:
            ctx.set_stream(torch.cuda.current_stream())
            ctx.set_inputs(torch.from_numpy(s.images).cuda(), torch.from_numpy(s.seg_prior).cuda(), None)
        else:
            ctx.set_inputs(s.images, s.seg_prior, None)
        return ctx.support_points()


FRAMES = [
    lambda: scenes.small_gray(0),
    lambda: scenes.small_gray(1, baselines=[-0.3, -0.1, 0.0, 0.2], D=24),
    lambda: scenes.small_gray(2, H=37, W=75, D=16),
    lambda: scenes.street_rgb(2, H=60, W=96, D=32, M=20),
    lambda: scenes.street_rgb(1, H=120, W=192, D=64, M=20),
    lambda: scenes.random_frame(4, scale=0.2),
    lambda: scenes.random_frame(7, scale=0.2),
]


@pytest.mark.parametrize("i", range(len(FRAMES)))
@pytest.mark.parametrize("grid", [4, 5])
def test_support_points_equal_oracle(i, grid):
    from paper_2003_11076_gb300 import lf
    s = FRAMES[i]()
    sp = lf.default_support_params(grid=grid, texture=60, window=2, min_support=1)
    got = _detect(s, sp)
    ref = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, _oracle_params(sp))
    assert ref["points"].shape[0] >= 5
    assert got.shape == ref["points"].shape
    assert np.array_equal(got, ref["points"].astype(np.float32))


def test_support_points_full_size_frame_and_device_inputs():
    from paper_2003_11076_gb300 import lf
    s = scenes.street_rgb(0)
    sp = lf.default_support_params()
    got = _detect(s, device=True)
    ref = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D, _oracle_params(sp))
    assert ref["points"].shape[0] > 5000
    assert np.array_equal(got, ref["points"].astype(np.float32))


def test_em_on_detected_support_points_matches_oracle():
    """The whole path from images alone: detected points -> prior -> EM,
    against the oracle run on the oracle's own support points."""
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(3)
    gp, op = params_pair()
    g = lf.run_scene(s, params=gp, detect_support=True)
    pts = O.support_points(s.images, s.seg_prior, s.baselines, s.d_min, s.d_max, s.D)["points"]
    assert np.array_equal(g["support_points"], pts.astype(np.float32))
    o = O.run(s.images, s.seg_prior, s.baselines, pts.astype(np.float32), s.d_min, s.d_max, s.D, s.iters,
              params=op)
    check_parity(g, o, what="EM on detected support points")
    # the detected prior is close to the ground-truth static disparity: within
    # the integer-shift resolution of the widest pair (1 / 0.2 = 5 candidates
    # per pixel, so half a pixel is 2.5 disparity units)
    mu = g["mu"]
    ok = ~np.isnan(mu)
    assert ok.mean() > 0.7
    assert np.median(np.abs(mu[ok] - s.gt_disparity[ok])) <= 2.5


def test_support_argument_checks():
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(0)
    with lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D) as ctx:
        for bad in (dict(grid=0), dict(ratio_pct=0), dict(ratio_pct=101), dict(texture=-1), dict(window=-1),
                    dict(delta=float("nan")), dict(min_support=-1)):
            with pytest.raises(lf.LfError) as e:
                ctx.set_support_params(lf.default_support_params(**bad))
            assert e.value.status == lf.LF_EINVAL
        assert ctx.support_points().shape == (0, 3)  # nothing detected yet
    cams = np.zeros((s.K, 3, 4), np.float32)
    for k, bk in enumerate(s.baselines):
        cams[k, :, :3] = np.eye(3)
        cams[k, 0, 3] = -bk
    with lf.Context(None, s.H, s.W, s.d_min, s.d_max, s.D, cameras=cams) as ctx:
        with pytest.raises(lf.LfError) as e:
            ctx.set_inputs(s.images, s.seg_prior, None)
        assert e.value.status == lf.LF_EINVAL and "rectified" in str(e.value)
