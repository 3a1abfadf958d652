"""The allocation-free sweep entry point, lf_run_em_static, through the C ABI.

It serves callers that cannot allocate device memory -- a framework whose own
memory pool owns the GPU and forbids raw cudaMalloc, or a latency-critical
loop that must not trigger the device-wide synchronisation cudaMalloc/cudaFree
can cause.  Given the same inputs and the prior map of the ordinary path, it
must reproduce lf_run_em's outputs within the parity tolerances of the other
GPU tests, on two calls in a row (all calls share one fixed scratch array
that keeps the previous call's contents).  The file is named so that pytest
collects it last; it needs nothing from the other tests.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

POST_TOL = 1e-4


def _static_call(lf, scene, mu_dev, torch):
    dev = torch.device("cuda")
    K, H, W = scene.K, scene.H, scene.W
    img = torch.from_numpy(np.ascontiguousarray(scene.images)).to(dev)
    seg = torch.from_numpy(np.ascontiguousarray(scene.seg_prior)).to(dev)
    out = {"d_idx": torch.full((H, W), -1, dtype=torch.int32, device=dev),
           "d": torch.full((H, W), float("nan"), dtype=torch.float32, device=dev),
           "post": torch.full((K, H, W), float("nan"), dtype=torch.float32, device=dev),
           "labels": torch.zeros((H, W), dtype=torch.int16, device=dev)}
    lf.run_em_static(scene.baselines, scene.d_min, scene.d_max, scene.D, scene.iters, img, seg, mu_dev, out,
                     stream=torch.cuda.current_stream())
    return {k: v.cpu().numpy() for k, v in out.items()}


def test_static_entry_matches_run_em_on_two_calls_in_a_row():
    import torch
    from paper_2003_11076_gb300 import build, lf, scenes
    assert torch.cuda.is_available()
    build.build()
    frames = [scenes.small_gray(0), scenes.street_rgb(3, H=72, W=96, D=32, iters=6, M=40)]
    for s in frames:  # two calls in a row, different sizes, D and input types
        ref = lf.run_scene(s)  # the ordinary entry point (allocates its buffers)
        mu = torch.from_numpy(ref["mu"]).cuda()
        got = _static_call(lf, s, mu, torch)
        assert np.array_equal(got["d_idx"], ref["d_idx"])
        assert np.array_equal(got["labels"].view(np.uint16), ref["labels"])
        assert np.array_equal(got["d"], ref["d"])
        assert np.max(np.abs(got["post"] - ref["post"])) <= POST_TOL


def test_static_entry_rejects_what_it_cannot_hold():
    import torch
    from paper_2003_11076_gb300 import build, lf, scenes
    build.build()
    s = scenes.small_gray(0)
    dev = torch.device("cuda")
    img = torch.from_numpy(s.images).to(dev)
    seg = torch.from_numpy(s.seg_prior).to(dev)
    mu = torch.zeros((s.H, s.W), dtype=torch.float32, device=dev)
    out = {"d_idx": torch.empty((s.H, s.W), dtype=torch.int32, device=dev)}
    with pytest.raises(lf.LfError) as e:  # more candidates than the scratch holds tables for
        lf.run_em_static(s.baselines, 0.0, 300.0, 301, 3, img, seg, mu, out)
    assert e.value.status == lf.LF_EINVAL and "256" in str(e.value)
    img_odd = torch.from_numpy(np.ascontiguousarray(s.images[:, :, :61])).to(dev)  # 244-byte rows
    seg_odd = torch.from_numpy(np.ascontiguousarray(s.seg_prior[:, :, :61])).to(dev)
    mu_odd = torch.zeros((s.H, 61), dtype=torch.float32, device=dev)
    out_odd = {"d_idx": torch.empty((s.H, 61), dtype=torch.int32, device=dev)}
    with pytest.raises(lf.LfError) as e:
        lf.run_em_static(s.baselines, s.d_min, s.d_max, s.D, 3, img_odd, seg_odd, mu_odd, out_odd)
    assert e.value.status == lf.LF_EINVAL and "aligned" in str(e.value)


def test_static_entry_checks_params_as_lf_create_does():
    """sigma = 0 or seg_threshold = 1 would make the sweep divide by zero or
    take log(thr / (1 - thr)) = inf; the call must refuse them, not return
    LF_OK with meaningless disparities."""
    import torch
    from paper_2003_11076_gb300 import build, lf, scenes
    build.build()
    s = scenes.small_gray(0)
    dev = torch.device("cuda")
    img = torch.from_numpy(s.images).to(dev)
    seg = torch.from_numpy(s.seg_prior).to(dev)
    mu = torch.zeros((s.H, s.W), dtype=torch.float32, device=dev)
    out = {"d_idx": torch.empty((s.H, s.W), dtype=torch.int32, device=dev)}
    for field, value in (("sigma", 0.0), ("seg_threshold", 1.0)):
        p = lf.default_params(**{field: value})
        with pytest.raises(lf.LfError) as e:
            lf.run_em_static(s.baselines, s.d_min, s.d_max, s.D, 3, img, seg, mu, out, params=p)
        assert e.value.status == lf.LF_EINVAL and field in str(e.value)
    # and a valid call right after still works
    ref = lf.run_scene(s)
    got = _static_call(lf, s, torch.from_numpy(ref["mu"]).cuda(), torch)
    assert np.array_equal(got["d_idx"], ref["d_idx"])
