"""GPU parity of the two EM variants (soft EM, joint MAP over (d, S)) against
the FP64 oracle, with the tolerances and excusal rule of the EM's own parity
tests; plus the argument checks of the modes."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_11076_gb300 import scenes
from test_gpu_parity import check_parity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2003_11076_gb300 import build
    build.build()
    O.build()


def _pair(mode, **kw):
    from paper_2003_11076_gb300 import lf
    gp = lf.default_params(em_mode=mode, **kw)
    op = O.Params(beta=float(np.float32(gp.beta)), gamma=float(np.float32(gp.gamma)),
                  sigma=float(np.float32(gp.sigma)), seg_threshold=float(np.float32(gp.seg_threshold)),
                  eps=float(np.float32(gp.eps)), mstep_seg_term=int(gp.mstep_seg_term), em_mode=mode)
    return gp, op


def _run_both(scene, mode, rows=None, iters=None, **kw):
    from paper_2003_11076_gb300 import lf
    gp, op = _pair(mode, **kw)
    g = lf.run_scene(scene, params=gp, iters=iters)
    o = O.run_scene(scene, params=op, rows=rows, iters=iters)
    return g, o


SOFT_FRAMES = [
    lambda: scenes.small_gray(0),
    lambda: scenes.small_gray(1),
    lambda: scenes.small_gray(2, H=37, W=75, M=12, D=16, iters=6),
    lambda: scenes.small_gray(3, baselines=[0.0], D=12, iters=3),
    lambda: scenes.small_gray(4, baselines=[-0.15, 0.0, 0.2], D=20, iters=5),
    lambda: scenes.small_gray(5, baselines=[-0.3, -0.15, 0.0, 0.1, 0.25, 0.4, 0.55], D=24, iters=4),
    lambda: scenes.small_gray(6, baselines=[-0.35, -0.25, -0.1, 0.0, 0.1, 0.2, 0.3, 0.45], D=16, iters=4),
    lambda: scenes.street_rgb(3, H=72, W=96, D=32, iters=6, M=40),
]


@pytest.mark.parametrize("i", range(len(SOFT_FRAMES)))
def test_soft_em_matches_oracle(i):
    s = SOFT_FRAMES[i]()
    g, o = _run_both(s, 1)
    check_parity(g, o, what=f"soft EM {s.name} K={s.K}")


@pytest.mark.parametrize("i", [0, 2, 3, 4, 5, 7])
def test_joint_map_matches_oracle(i):
    s = SOFT_FRAMES[i]()
    g, o = _run_both(s, 2)
    check_parity(g, o, what=f"joint MAP {s.name} K={s.K}")
    from paper_2003_11076_gb300 import lf
    assert g["stats"]["nominal_ray_samples"] == s.H * s.W * s.K * s.D  # one sweep, iterations unused


def test_joint_map_twelve_cameras():
    b = [-0.3, -0.25, -0.2, -0.15, -0.1, -0.05, 0.0, 0.05, 0.1, 0.15, 0.2, 0.25]
    s = scenes.small_gray(7, baselines=b, H=20, W=40, D=8, iters=2, M=12)
    g, o = _run_both(s, 2)
    check_parity(g, o, what="joint MAP K=12")


def test_soft_em_full_frame():
    """The 960x600 RGB frame in soft-EM mode, every pixel against the oracle."""
    s = scenes.street_rgb(0)
    g, o = _run_both(s, 1)
    check_parity(g, o, what="soft EM street_rgb")


def test_joint_map_full_frame():
    """The 960x600 RGB frame in joint-MAP mode, every pixel against the oracle."""
    s = scenes.street_rgb(0)
    g, o = _run_both(s, 2)
    check_parity(g, o, what="joint MAP street_rgb")


def test_variants_differ_from_hard_em_and_bound_it():
    """The modes are different algorithms (some pixel's result differs), and
    the joint MAP objective bounds the hard EM's final objective."""
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(1)
    hard = lf.run_scene(s)
    soft = lf.run_scene(s, params=lf.default_params(em_mode=1))
    joint = lf.run_scene(s, params=lf.default_params(em_mode=2))
    assert not (np.array_equal(hard["d_idx"], soft["d_idx"]) and np.array_equal(hard["labels"], soft["labels"])
                and np.array_equal(hard["post"], soft["post"]))
    assert not (np.array_equal(hard["d_idx"], joint["d_idx"]) and np.array_equal(hard["labels"], joint["labels"]))
    o_joint = O.run_scene(s, params=O.Params(em_mode=2), iters=1)
    o_hard = O.run_scene(s)
    assert np.all(o_hard["J_t"][-1] <= o_joint["J_t"][0] + 1e-9)


@pytest.mark.parametrize("mode", [1, 2])
def test_variant_dynamic_only_equals_full_mode_on_dynamic_pixels(mode):
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(0)
    full = lf.run_scene(s, params=lf.default_params(em_mode=mode))
    dyn = lf.run_scene(s, params=lf.default_params(em_mode=mode, dynamic_only=1))
    ref = int(np.argmin(np.abs(s.baselines)))
    m = s.seg_prior[ref] >= np.float32(0.7)
    assert 0 < m.sum() < m.size
    for k in ("d_idx", "labels", "d", "refocus"):
        assert np.array_equal(dyn[k][m], full[k][m]), k
    assert np.array_equal(dyn["post"][:, m], full["post"][:, m])
    assert np.all(np.isnan(dyn["post"][:, ~m])) and np.all(dyn["labels"][~m] == 0)


@pytest.mark.parametrize("make", [
    lambda: scenes.small_gray(2),
    lambda: scenes.street_rgb(0),
    lambda: scenes.small_gray(16, D=7),
    lambda: scenes.small_gray(17, baselines=[-0.35, -0.25, -0.15, -0.05, 0.0, 0.1, 0.2, 0.3], D=40),
])
def test_soft_em_early_exit_is_exact(make):
    """With the early exit only the pixels still iterating run, regrouped into
    dense warps and, once few are left, one warp per pixel; without it every
    pixel runs every iteration.  Both give the same bits."""
    from paper_2003_11076_gb300 import lf
    s = make()
    a = lf.run_scene(s, params=lf.default_params(em_mode=1, early_exit=1), iters=8)
    b = lf.run_scene(s, params=lf.default_params(em_mode=1, early_exit=0), iters=8)
    for k in ("d_idx", "labels", "d", "post", "refocus"):
        assert np.array_equal(a[k], b[k]), k
    assert a["stats"]["executed_ray_samples"] < b["stats"]["executed_ray_samples"]


def test_variant_argument_checks():
    import torch
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(0)
    nine = [-0.4, -0.3, -0.2, -0.1, 0.0, 0.1, 0.2, 0.3, 0.4]
    with pytest.raises(lf.LfError) as e:
        lf.Context(nine, 16, 32, 0.0, 8.0, 8, lf.default_params(em_mode=1))
    assert e.value.status == lf.LF_EINVAL and "8 cameras" in str(e.value)
    with pytest.raises(lf.LfError) as e:
        lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D, lf.default_params(em_mode=2, precision=1))
    assert e.value.status == lf.LF_EINVAL
    with pytest.raises(lf.LfError) as e:
        lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D, lf.default_params(em_mode=3))
    assert e.value.status == lf.LF_EINVAL
    with pytest.raises(lf.LfError) as e:
        lf.Batch(lf.default_params(em_mode=1))
    assert e.value.status == lf.LF_EINVAL
    dev = torch.device("cuda")
    out = {"d_idx": torch.empty((s.H, s.W), dtype=torch.int32, device=dev)}
    with pytest.raises(lf.LfError) as e:
        lf.run_em_static(s.baselines, s.d_min, s.d_max, s.D, 3, torch.from_numpy(s.images).to(dev),
                         torch.from_numpy(s.seg_prior).to(dev), torch.zeros((s.H, s.W), device=dev), out,
                         params=lf.default_params(em_mode=2))
    assert e.value.status == lf.LF_EINVAL
