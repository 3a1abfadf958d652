"""Host-side arithmetic of the benchmark line (CPU only): the op models the
ALU roofline divides by, and the HBM roofline's bytes and peak."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_scope_op_model_per_unit():
    """29 per static ray sample, 4 per dynamic one, 12 per (pixel, candidate),
    20 per E-step label vector: one pixel-iteration of five cameras and 64
    candidates with 70 % static samples."""
    K, D = 5, 64
    samples = K * D
    static = 0.7 * samples
    ops = bench.scope_ops(samples, static, D, 1, K)
    assert ops == pytest.approx(29 * static + 4 * (samples - static) + 12 * D + 20 * 32)


def test_tight_model_equals_the_full_sweep_count_without_pruning():
    """Over a full sweep (D objectives per pixel-iteration) the tight model is
    the per-pixel-iteration count of the unpruned kernel."""
    for K, D in ((1, 1), (5, 64), (9, 128)):
        assert bench.tight_ops(D * 7, 7, K) == 7 * bench.sweep_ops_per_pixel_iter(K, D)


def test_hbm_roofline_uses_the_measured_copy_bandwidth(tmp_path):
    peaks = tmp_path / "peaks.json"
    peaks.write_text(json.dumps({"hbm_gbs": 5000.0}))
    r = bench.hbm_roofline(40e6, 0.25e-3, str(peaks))
    assert r["bound"] == "hbm" and r["unit"] == "GB/s"
    assert r["achieved"] == pytest.approx(160.0)
    assert r["peak"] == 5000.0 and r["frac"] == pytest.approx(160.0 / 5000.0)
    assert r["peak_basis"].startswith("of measured")


@pytest.mark.parametrize("content", [None, "{}", "not json", json.dumps({"hbm_gbs": 0})])
def test_hbm_roofline_falls_back_without_a_measurement(tmp_path, content):
    peaks = tmp_path / "peaks.json"
    if content is not None:
        peaks.write_text(content)
    r = bench.hbm_roofline(6.8e12, 1.0, str(peaks))
    assert r["peak"] == bench.HBM_FALLBACK_GBS and r["frac"] == pytest.approx(1.0)
    assert r["peak_basis"].startswith("of fallback")


def test_traffic_record_parses():
    """The recorded ncu traffic of the sweep kernel carries the source hash it
    was taken at and a per-launch byte count equal to read + write."""
    kv = {}
    for line in open(bench.TRAFFIC_FILE):
        if "=" in line and not line.lstrip().startswith("#"):
            k, v = line.split("=", 1)
            kv[k.strip()] = v.strip()
    assert len(kv["kernel_sha"]) == 16
    assert int(kv["dram_bytes_per_launch"]) == int(kv["dram_bytes_read"]) + int(kv["dram_bytes_write"])
