"""Reduced-precision storage (float16 / bfloat16 staged maps and images,
float32 arithmetic) against the FP64 oracle, beside the float32 GPU path.

Each case prints one report line: disparity-index agreement, posterior max
error and refocus max / mean absolute error (posteriors and refocus on the
pixels where disparity and labels agree with the oracle).  The assertions are
the accuracy this storage is expected to keep.
"""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_11076_gb300 import scenes

pytestmark = pytest.mark.gpu

NAMES = {0: "f32", 1: "f16", 2: "bf16"}
# minimum disparity-index agreement with the oracle per storage type
MIN_AGREE = {0: 0.999, 1: 0.97, 2: 0.85}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_11076_gb300 import build
    build.build()
    O.build()


def _oracle_params(gp):
    return O.Params(beta=float(np.float32(gp.beta)), gamma=float(np.float32(gp.gamma)),
                    sigma=float(np.float32(gp.sigma)), seg_threshold=float(np.float32(gp.seg_threshold)),
                    eps=float(np.float32(gp.eps)), mstep_seg_term=int(gp.mstep_seg_term))


def report(scene, prec, rows=None):
    from paper_2003_11076_gb300 import lf
    gp = lf.default_params(precision=prec)
    g = lf.run_scene(scene, params=gp)
    o = O.run_scene(scene, params=_oracle_params(gp), rows=rows)
    sl = slice(None) if rows is None else slice(*rows)
    same = g["d_idx"][sl] == o["d_idx"][sl]
    agree = same & (g["labels"][sl] == o["labels"][sl])
    post_err = np.abs(g["post"][:, sl] - o["post"][:, sl])[:, agree]
    ref_err = np.abs(g["refocus"][sl] - o["refocus"][sl])[agree]
    r = {"scene": scene.name, "size": f"{scene.W}x{scene.H}", "precision": NAMES[prec],
         "d_agreement": float(same.mean()), "labels_agreement": float(agree.mean()),
         "posterior_max_err": float(post_err.max()) if post_err.size else 0.0,
         "refocus_max_err": float(ref_err.max()) if ref_err.size else 0.0,
         "refocus_mean_err": float(ref_err.mean()) if ref_err.size else 0.0}
    print("PRECISION_REPORT " + json.dumps(r))
    return r


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_small_gray_precision(prec):
    r = report(scenes.small_gray(0), prec)
    assert r["d_agreement"] >= MIN_AGREE[prec]
    assert r["refocus_mean_err"] <= (1e-4 if prec == 0 else 1e-2)


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_street_rgb_precision_sampled_rows(prec):
    """The paper-shaped RGB frame at full size; the oracle checks one band."""
    r = report(scenes.street_rgb(0), prec, rows=(296, 304))
    assert r["d_agreement"] >= MIN_AGREE[prec]
    assert r["refocus_mean_err"] <= (1e-4 if prec == 0 else 1e-2)


def test_half_precision_image_inputs():
    """float16 / bfloat16 images are accepted as inputs (read by TMA as is)."""
    import torch
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(1)
    base = lf.run_scene(s, params=lf.default_params(precision=1))
    with lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D, lf.default_params(precision=1)) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        img16 = torch.from_numpy(s.images).cuda().to(torch.float16).contiguous()
        ctx.set_inputs(img16, torch.from_numpy(s.seg_prior).cuda(), s.points)
        out = ctx.run(s.iters, device=True)
        ctx.synchronize()
    # the float32 input converted on the device equals the float16 input
    assert np.array_equal(out["d_idx"].cpu().numpy(), base["d_idx"])
