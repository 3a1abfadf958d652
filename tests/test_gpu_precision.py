"""Reduced-precision storage of the staged maps (float32 arithmetic) against
the FP64 oracle, beside the float32 GPU path.

Storage per mode: float16 and bfloat16 keep the Sobel responses in 16 bits;
the luminance and the log segmentation maps are float32 in every mode
(16-bit luminance alone costs 0.16 % / 1.2 % of the disparity agreement on
the float32 gray frames, bfloat16 log maps 0.06 % on the 960 x 600 frame),
and input images stay in the type the caller gives.

The contract: the disparity index equal on at least 99.9 % of the pixels and
every mismatch at a pixel the oracle itself cannot decide robustly (excused).
float32 and float16 storage meet both parts.  bfloat16 meets the 99.9 % floor
but not the second part everywhere: its 8-bit significand moves the
photometric term of a few pixels by more than the float32 tie threshold, so
for it the pixels beyond that threshold are reported and only bounded (at
most 1 in 10,000), which is the part of the contract it cannot reach.

Each case prints one report line: disparity-index agreement, mismatches not
excused by the float32 rule, posterior max error and refocus max / mean
absolute error (posteriors and refocus on the pixels where disparity and
labels agree with the oracle).
"""
import json

import numpy as np
import pytest

from oracle import oracle as O
from paper_2003_11076_gb300 import scenes

pytestmark = pytest.mark.gpu

NAMES = {0: "f32", 1: "f16", 2: "bf16"}
D_FRAC = 0.999


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2003_11076_gb300 import build
    build.build()
    O.build()


def _oracle_params(gp):
    return O.Params(beta=float(np.float32(gp.beta)), gamma=float(np.float32(gp.gamma)),
                    sigma=float(np.float32(gp.sigma)), seg_threshold=float(np.float32(gp.seg_threshold)),
                    eps=float(np.float32(gp.eps)), mstep_seg_term=int(gp.mstep_seg_term))


def _compare(g, o):
    exc = O.excused(o)
    same = g["d_idx"] == o["d_idx"]
    agree = same & (g["labels"] == o["labels"])
    post_err = np.abs(g["post"] - o["post"])[:, agree]
    ref_err = np.abs(g["refocus"] - o["refocus"])[agree]
    return {"pixels": int(same.size), "d_mismatch": int((~same).sum()),
            "non_excused": int((~agree & ~exc).sum()),
            "post_max": float(post_err.max()) if post_err.size else 0.0,
            "ref_max": float(ref_err.max()) if ref_err.size else 0.0,
            "ref_sum": float(ref_err.sum()), "ref_n": int(ref_err.size)}


def report(frames, prec, name):
    """Run every frame at storage `prec` on the GPU and in the oracle; one
    report over all their pixels."""
    from paper_2003_11076_gb300 import lf
    gp = lf.default_params(precision=prec)
    tot = None
    for s in frames:
        c = _compare(lf.run_scene(s, params=gp), O.run_scene(s, params=_oracle_params(gp)))
        if tot is None:
            tot = c
        else:
            for k in ("pixels", "d_mismatch", "non_excused", "ref_sum", "ref_n"):
                tot[k] += c[k]
            tot["post_max"] = max(tot["post_max"], c["post_max"])
            tot["ref_max"] = max(tot["ref_max"], c["ref_max"])
    r = {"scene": name, "frames": len(frames), "precision": NAMES[prec],
         "d_agreement": 1.0 - tot["d_mismatch"] / tot["pixels"], "non_excused_mismatches": tot["non_excused"],
         "posterior_max_err": tot["post_max"], "refocus_max_err": tot["ref_max"],
         "refocus_mean_err": tot["ref_sum"] / max(tot["ref_n"], 1)}
    print("PRECISION_REPORT " + json.dumps(r))
    return r


def _assert_contract(r, pixels):
    assert r["d_agreement"] >= D_FRAC, r
    if r["precision"] == "bf16":
        assert r["non_excused_mismatches"] <= 1e-4 * pixels, r
    else:
        assert r["non_excused_mismatches"] == 0, r
    assert r["posterior_max_err"] <= (1e-4 if r["precision"] == "f32" else 5e-3), r
    assert r["refocus_max_err"] <= 1e-3, r


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_small_gray_precision(prec):
    """Four 64 x 48 float32 gray frames (12,288 pixels)."""
    frames = [scenes.small_gray(i) for i in range(4)]
    _assert_contract(report(frames, prec, "small_gray x4"), sum(f.H * f.W for f in frames))


@pytest.mark.parametrize("prec", [0, 1, 2])
def test_street_rgb_precision_full_frame(prec):
    """The paper-shaped 960 x 600 RGB frame, every pixel."""
    s = scenes.street_rgb(0)
    _assert_contract(report([s], prec, "street_rgb"), s.H * s.W)


@pytest.mark.parametrize("prec", [0, 1])
def test_half_precision_image_inputs(prec):
    """float16 images are accepted as inputs (read by TMA as they are).  The
    oracle gets the same image values (the float16 numbers, widened); the
    float16 input gives the same bits as those values passed as float32."""
    import torch
    from paper_2003_11076_gb300 import lf
    s = scenes.small_gray(1)
    s.images = s.images.astype(np.float16).astype(np.float32)  # the values a float16 caller holds
    gp = lf.default_params(precision=prec)
    base = lf.run_scene(s, params=gp)
    with lf.Context(s.baselines, s.H, s.W, s.d_min, s.d_max, s.D, gp) as ctx:
        ctx.set_stream(torch.cuda.current_stream())
        img16 = torch.from_numpy(s.images).cuda().to(torch.float16).contiguous()
        ctx.set_inputs(img16, torch.from_numpy(s.seg_prior).cuda(), s.points)
        out = ctx.run(s.iters, device=True)
        ctx.synchronize()
    for k in ("d_idx", "post", "refocus"):
        assert np.array_equal(out[k].cpu().numpy(), base[k]), k
    c = _compare(base, O.run_scene(s, params=_oracle_params(gp)))
    assert c["d_mismatch"] <= (1 - D_FRAC) * c["pixels"] and c["non_excused"] == 0, c
