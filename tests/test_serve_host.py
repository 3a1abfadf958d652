"""Host logic of the request loop (CPU only)."""
import numpy as np

from paper_2003_11076_gb300 import scenes, serve


def test_poisson_arrivals_rate_and_order():
    t = serve.poisson_arrivals(200.0, 20.0, seed=3)
    assert np.all(np.diff(t) > 0) and t[0] >= 0 and t[-1] < 20.0
    assert abs(len(t) / 20.0 - 200.0) < 4 * np.sqrt(200.0 * 20.0) / 20.0
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 200.0) < 0.1 / 200.0       # exponential gaps
    assert abs(np.std(gaps) / gaps.mean() - 1.0) < 0.1


def test_percentiles():
    lat = list(np.linspace(0.001, 0.1, 100))
    p = serve.percentiles(lat)
    assert abs(p["p50_ms"] - 50.5) < 1e-9 and p["p99_ms"] > p["p95_ms"] > p["p50_ms"]
    assert serve.percentiles([])["p50_ms"] is None


def test_request_device_bytes_cover_inputs_and_outputs():
    s = scenes.small_gray(0)
    r = serve.Request.from_scene(7, s, arrival=0.25)
    need = r.device_bytes()
    HW = s.H * s.W
    assert need >= s.images.nbytes + s.seg_prior.nbytes + HW * (4 + 4 + 2) + s.K * HW * 4 + HW * 4
    assert (r.K, r.H, r.W, r.C) == (s.K, s.H, s.W, 1) and r.arrival == 0.25
