"""GPU parity of the calibrated (non-rectified) array path -- Eq. 1 with a
3x4 matrix per camera, bilinear sampling -- against the FP64 oracle, with the
tolerances and excusal rule of the rectified parity tests."""
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


def _run_both(s, rows=None, **kw):
    from paper_2003_11076_gb300 import lf
    gp, op = params_pair(**kw)
    g = lf.run_scene(s, params=gp)
    o = O.run_scene(s, params=op, rows=rows)
    return g, o


FRAMES = [
    lambda: scenes.small_gray(0, calibrated=True),
    lambda: scenes.small_gray(1, calibrated=True, rot_deg=3.0),
    lambda: scenes.small_gray(2, calibrated=True, H=37, W=75, M=12, D=16, iters=6),
    lambda: scenes.small_gray(3, calibrated=True, baselines=[0.0, 0.15, 0.3], D=20),
    lambda: scenes.small_gray(4, calibrated=True, baselines=[-0.3, -0.15, 0.0, 0.1, 0.25, 0.4, 0.55], D=24,
                              iters=4),
    lambda: scenes.small_gray(5, calibrated=True, H=20, W=40, D=8, iters=3, M=12,
                              baselines=[-0.3, -0.25, -0.2, -0.15, -0.1, -0.05, 0.0, 0.05, 0.1, 0.15, 0.2, 0.25]),
    lambda: scenes.street_rgb(3, calibrated=True, H=72, W=96, D=32, iters=6, M=40, rot_deg=1.5),
]


@pytest.mark.parametrize("i", range(len(FRAMES)))
def test_calibrated_frame_matches_oracle(i):
    s = FRAMES[i]()
    assert s.cameras is not None
    g, o = _run_both(s)
    check_parity(g, o, what=f"calibrated {s.name} K={s.K}")
    assert g["stats"]["kernels_launched"] == 4  # prior, descriptor maps, sweep, refocus


def test_calibrated_full_frame():
    """The 960x600 RGB street frame seen by a non-rectified array (rotations
    up to 0.6 degrees: shifts of up to 12 px in both directions), every pixel
    against the oracle."""
    s = scenes.street_rgb(0, calibrated=True)
    g, o = _run_both(s)
    check_parity(g, o, what="calibrated street_rgb")


def test_rectified_matrices_agree_with_the_rectified_path():
    """[I | (-b_k, 0, 0)] through lf_create_calibrated and the baselines
    through lf_create both match the oracle, and each other on all but the
    pixels whose arg-max the float32 rounding of the ray position can flip."""
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(1)
    cams = np.zeros((s.K, 3, 4), np.float32)
    for k, bk in enumerate(s.baselines):
        cams[k, :, :3] = np.eye(3)
        cams[k, 0, 3] = -bk
    rect = lf.run_scene(s)
    s.cameras = cams
    gen = lf.run_scene(s)
    o = O.run_scene(s)
    gp, _ = params_pair()
    check_parity(gen, o, what="rectified matrices")
    assert np.mean(gen["d_idx"] == rect["d_idx"]) >= 0.999


def test_calibrated_dynamic_only_and_median():
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(0, calibrated=True)
    full = lf.run_scene(s)
    dyn = lf.run_scene(s, params=lf.default_params(dynamic_only=1))
    m = s.seg_prior[s.ref] >= np.float32(0.7)
    assert 0 < m.sum() < m.size
    for k in ("d_idx", "labels", "d", "refocus"):
        assert np.array_equal(dyn[k][m], full[k][m]), k
    assert np.array_equal(dyn["post"][:, m], full["post"][:, m])
    assert np.all(np.isnan(dyn["post"][:, ~m])) and np.all(dyn["labels"][~m] == 0)
    img = s.images[s.ref].astype(np.float32)
    assert np.max(np.abs(dyn["refocus"][~m] - img[~m])) <= 1e-6
    assert dyn["stats"]["executed_ray_samples"] < full["stats"]["executed_ray_samples"]
    med = lf.run_scene(s, params=lf.default_params(median=1))
    assert np.allclose(med["refocus"], O.median3(full["refocus"].astype(np.float64)), atol=1e-6)


def test_calibrated_device_io_and_early_exit():
    import torch
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(2, calibrated=True)
    host = lf.run_scene(s)
    with lf.Context(None, s.H, s.W, s.d_min, s.d_max, s.D, cameras=s.cameras) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        ctx.set_inputs(torch.from_numpy(s.images).cuda(), torch.from_numpy(s.seg_prior).cuda(), s.points)
        out = ctx.run(s.iters, device=True)
        ctx.synchronize()
    for k in ("d_idx", "d", "post", "refocus"):
        assert np.array_equal(out[k].cpu().numpy(), host[k]), k
    slow = lf.run_scene(s, params=lf.default_params(early_exit=0))
    for k in ("d_idx", "labels", "d", "post", "refocus"):
        assert np.array_equal(slow[k], host[k]), k
    assert host["stats"]["executed_ray_samples"] < slow["stats"]["executed_ray_samples"]


PRUNE_FRAMES = FRAMES + [
    lambda: scenes.street_rgb(0, calibrated=True),
    lambda: scenes.small_gray(6, calibrated=True, rot_deg=2.0),
]


@pytest.mark.parametrize("i", range(len(PRUNE_FRAMES)))
def test_calibrated_pruning_is_exact(i):
    """Candidate pruning of the calibrated sweep (bound: log prior + 0, every
    log probability being <= 0) gives the full sweeps' bits, one to twelve
    cameras."""
    from paper_2003_11076_gb300 import lf
    s = PRUNE_FRAMES[i]()
    a = lf.run_scene(s, params=lf.default_params(prune=1))
    b = lf.run_scene(s, params=lf.default_params(prune=0))
    for k in ("d_idx", "d", "labels", "post", "refocus"):
        assert np.array_equal(a[k], b[k], equal_nan=True), k
    assert a["stats"]["executed_pixel_iterations"] == b["stats"]["executed_pixel_iterations"]
    assert b["stats"]["executed_ray_samples"] == s.K * s.D * b["stats"]["executed_pixel_iterations"]
    # each bounded M-step costs one extra objective (the bound's reference
    # candidate); with more than a few candidates the bound saves far more
    assert a["stats"]["executed_ray_samples"] <= b["stats"]["executed_ray_samples"] + \
        s.K * a["stats"]["executed_pixel_iterations"]
    if s.D >= 16:
        assert a["stats"]["executed_ray_samples"] < b["stats"]["executed_ray_samples"]
