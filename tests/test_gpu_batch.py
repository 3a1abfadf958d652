"""Uneven batches (lf_batch_*): every frame's result in the mix equals its
result run alone through lf_run_em, and a batch whose contents change but
whose shape does not replays its captured CUDA graph."""
import numpy as np
import pytest

from paper_2003_11076_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_11076_gb300 import build
    build.build()


def _frames():
    # different sizes, camera counts, D, iterations and input types
    out = [scenes.small_gray(0),
           scenes.small_gray(1, H=37, W=75, M=12, D=16, iters=3),
           scenes.small_gray(2, baselines=[-0.3, -0.15, 0.0, 0.1, 0.25, 0.4, 0.55], D=24, iters=4),
           scenes.street_rgb(0, H=72, W=96, D=32, iters=6, M=40),
           scenes.small_gray(3, baselines=[0.0, 0.2, 0.4], H=20, W=130, D=40, iters=7)]
    out.append(scenes.random_frame(0, scale=0.25))
    return out


def _run_batch(lf, torch, frames, batch=None, params=None):
    b = batch or lf.Batch(params)
    b.set_stream(torch.cuda.current_stream())
    outs = []
    for s in frames:
        o = lf.device_outputs(s.K, s.H, s.W, s.C)
        b.add(s.baselines, s.d_min, s.d_max, s.D, s.iters, torch.from_numpy(s.images).cuda(),
              torch.from_numpy(s.seg_prior).cuda(), s.points, o)
        outs.append(o)
    b.run()
    b.synchronize()
    return b, [{k: v.cpu().numpy() for k, v in o.items()} for o in outs]


def _assert_same(alone, mixed):
    assert np.array_equal(mixed["d_idx"], alone["d_idx"])
    assert np.array_equal(mixed["labels"].view(np.uint16), alone["labels"])
    assert np.array_equal(mixed["d"], alone["d"])
    assert np.max(np.abs(mixed["post"] - alone["post"])) <= 1e-6
    assert np.max(np.abs(mixed["refocus"] - alone["refocus"])) <= 1e-6


def test_batch_results_equal_single_frame_results():
    import torch
    from paper_2003_11076_gb300 import lf
    frames = _frames()
    b, got = _run_batch(lf, torch, frames)
    st = b.stats()
    for s, g in zip(frames, got):
        _assert_same(lf.run_scene(s), g)
    assert st["runs"] == 1 and st["graph_captures"] == 1
    assert st["nominal_ray_samples"] == sum(s.nominal_ray_samples for s in frames)
    assert 0 < st["executed_ray_samples"] <= st["nominal_ray_samples"]
    b.close()


def test_batch_graph_is_replayed_when_only_contents_change():
    import torch
    from paper_2003_11076_gb300 import lf
    frames = _frames()
    b, first = _run_batch(lf, torch, frames)
    # same shapes, new pixel data (other noise draws / priors)
    frames2 = [scenes.small_gray(10), scenes.small_gray(11, H=37, W=75, M=12, D=16, iters=3),
               scenes.small_gray(12, baselines=[-0.3, -0.15, 0.0, 0.1, 0.25, 0.4, 0.55], D=24, iters=4),
               scenes.street_rgb(5, H=72, W=96, D=32, iters=6, M=40),
               scenes.small_gray(13, baselines=[0.0, 0.2, 0.4], H=20, W=130, D=40, iters=7),
               scenes.random_frame(0, scale=0.25)]
    b.clear()
    b, second = _run_batch(lf, torch, frames2, batch=b)
    st = b.stats()
    for s, g in zip(frames2, second):
        _assert_same(lf.run_scene(s), g)
    assert st["graph_captures"] == 1
    b.close()


def test_batch_reduced_precision_matches_single_frame():
    import torch
    from paper_2003_11076_gb300 import lf
    p = lf.default_params(precision=1)
    frames = _frames()[:4]
    b, got = _run_batch(lf, torch, frames, params=p)
    for s, g in zip(frames, got):
        _assert_same(lf.run_scene(s, params=lf.default_params(precision=1)), g)
    b.close()


def test_empty_batch_is_an_error():
    from paper_2003_11076_gb300 import lf
    with lf.Batch() as b:
        with pytest.raises(lf.LfError) as e:
            b.run()
        assert e.value.status == lf.LF_ESTATE


# Frames of the uneven-batch workload itself (random_frame(i), the generator
# the batch benchmark draws from): the largest (1269 x 1019, K = 5, D = 128),
# the widest disparity halo (K = 9, D = 128, 109 columns each side), a tall
# nine-camera frame (705 x 969), K = 7 at D = 128 and D = 32, and K = 3.
ORACLE_FRAMES = (49, 42, 45, 19, 8, 25)


def test_batch_frames_match_the_oracle():
    """The persistent batch kernel (per-frame descriptors in global memory,
    nine-camera launch group, wide halos, autotuned tiles) against the FP64
    oracle on every pixel of uneven workload frames, with the parity rule of
    the single-frame tests."""
    import torch
    from oracle import oracle as O
    from paper_2003_11076_gb300 import lf
    from test_gpu_parity import check_parity, params_pair
    O.build()
    frames = [scenes.random_frame(i) for i in ORACLE_FRAMES]
    assert {s.K for s in frames} == {3, 5, 7, 9} and max(s.D for s in frames) == 128
    gp, op = params_pair()
    b = lf.Batch(gp, autotune=True)
    b, got = _run_batch(lf, torch, frames, batch=b)
    for i, s, g in zip(ORACLE_FRAMES, frames, got):
        g = dict(g)
        g["labels"] = g["labels"].view(np.uint16)
        o = O.run_scene(s, params=op)
        frac, exc = check_parity(g, o, what=f"random_frame({i}) {s.W}x{s.H} K={s.K} D={s.D}")
        print(f"random_frame({i}) {s.W}x{s.H} K={s.K} D={s.D}: agreement {frac:.6f}, excused {exc:.5f}")
    b.close()
