"""Failure handling without a GPU fault: device allocations made to fail on
the host (lf_inject_alloc_failure) come back as LF_ENOMEM, leave no context
half-made, and the same context or batch works again on the next call."""
import ctypes

import numpy as np
import pytest

from paper_2003_11076_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True)
def _lib():
    from paper_2003_11076_gb300 import build, lf
    build.build()
    yield lf
    lf.load().lf_inject_alloc_failure(-1)  # never leave the injection armed


def test_create_reports_enomem_and_returns_no_context(_lib):
    lf = _lib
    s = scenes.small_gray(0)
    b = np.ascontiguousarray(s.baselines, np.float32)
    for after in (0, 2, 5):  # the first, third and sixth of lf_create's allocations
        lf.load().lf_inject_alloc_failure(after)
        h = ctypes.c_void_p()
        st = lf.load().lf_create(ctypes.byref(h), s.K, b.ctypes.data, s.H, s.W, s.d_min, s.d_max, s.D, None)
        assert st == lf.LF_ENOMEM and not h.value
        assert "out of device memory" in lf.load().lf_last_error(None).decode()
    lf.load().lf_inject_alloc_failure(-1)
    out = lf.run_scene(s)  # nothing was left half-made
    assert out["d_idx"].shape == (s.H, s.W)


def test_run_with_host_outputs_recovers_after_enomem(_lib):
    lf = _lib
    s = scenes.small_gray(1)
    ref = lf.run_scene(s)
    with lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D) as ctx:
        ctx.set_inputs(s.images, s.seg_prior, s.points)
        lf.load().lf_inject_alloc_failure(0)  # the first output staging buffer
        with pytest.raises(lf.LfError) as e:
            ctx.run(s.iters)
        assert e.value.status == lf.LF_ENOMEM
        out = ctx.run(s.iters)  # the same context, the injection spent
        for k in ("d_idx", "labels", "post", "refocus"):
            assert np.array_equal(out[k], ref[k]), k
        rgb = np.ascontiguousarray(np.repeat(s.images[..., None], 3, axis=3))  # three times the staging bytes
        lf.load().lf_inject_alloc_failure(0)  # the larger input staging buffer
        with pytest.raises(lf.LfError) as e:
            ctx.set_inputs(rgb, s.seg_prior, s.points)
        assert e.value.status == lf.LF_ENOMEM
        with pytest.raises(lf.LfError) as e:  # no inputs any more: call order enforced
            ctx.run(s.iters)
        assert e.value.status == lf.LF_ESTATE
        ctx.set_inputs(s.images, s.seg_prior, s.points)
        assert np.array_equal(ctx.run(s.iters)["d_idx"], ref["d_idx"])


def test_batch_run_recovers_after_enomem(_lib):
    import torch
    lf = _lib
    frames = [scenes.small_gray(0), scenes.small_gray(2, H=37, W=75, M=12, D=16, iters=3)]

    def add_all(b):
        outs = []
        for s in frames:
            o = lf.device_outputs(s.K, s.H, s.W, s.C)
            b.add(s.baselines, s.d_min, s.d_max, s.D, s.iters, torch.from_numpy(s.images).cuda(),
                  torch.from_numpy(s.seg_prior).cuda(), s.points, o)
            outs.append(o)
        return outs

    with lf.Batch() as b:
        b.set_stream(torch.cuda.current_stream())
        add_all(b)
        lf.load().lf_inject_alloc_failure(0)
        with pytest.raises(lf.LfError) as e:
            b.run()
        assert e.value.status == lf.LF_ENOMEM
        b.clear()
        outs = add_all(b)
        b.run()
        b.synchronize()
        for s, o in zip(frames, outs):
            assert np.array_equal(o["d_idx"].cpu().numpy(), lf.run_scene(s)["d_idx"])
