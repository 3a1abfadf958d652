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


def test_arena_first_fit_merges_and_never_overlaps():
    """The server's block allocator: aligned first-fit, freed neighbours
    merge back into one range, live ranges never overlap, and a request
    larger than the block never fits."""
    a = serve.Arena(4096, align=256)
    offs = [a.alloc(300), a.alloc(256), a.alloc(1000)]
    assert offs == [0, 512, 768] and a.bytes_used == 512 + 256 + 1024
    assert a.alloc(4096) is None and not a.fits_ever(4097) and a.fits_ever(4096)
    a.free(512)
    assert a.alloc(200) == 512            # first fit reuses the hole
    a.free(0)
    a.free(512)
    a.free(768)
    assert a.free_list == [(0, 4096)] and a.bytes_used == 0
    rng = np.random.default_rng(0)
    live = {}
    for _ in range(2000):
        if live and rng.random() < 0.45:
            off = list(live)[rng.integers(len(live))]
            a.free(off)
            del live[off]
        else:
            n = int(rng.integers(1, 900))
            off = a.alloc(n)
            if off is not None:
                live[off] = a.size_of(n)
        spans = sorted(live.items())
        assert all(o1 + s1 <= o2 for (o1, s1), (o2, _) in zip(spans, spans[1:]))
        assert all(o % 256 == 0 and o + s <= 4096 for o, s in spans)
        assert a.bytes_used == sum(live.values())
        assert sum(s for _, s in a.free_list) == 4096 - a.bytes_used


def test_request_output_layout_and_bytes():
    s = scenes.street_rgb(0, H=40, W=50, D=16, iters=3, M=10)
    r = serve.Request.from_scene(1, s)
    names = [n for n, _, _ in r.output_layout()]
    assert names == ["d_idx", "d", "post", "labels", "refocus"]
    assert dict((n, sh) for n, sh, _ in r.output_layout())["refocus"] == (40, 50, 3)
    assert r.output_bytes() % 256 == 0 and r.device_bytes() > r.output_bytes()


def test_arena_peak_is_the_largest_bytes_in_use():
    """The server reports the device block's peak use: the largest sum of live
    (aligned) ranges, which frees do not lower."""
    a = serve.Arena(8192, align=256)
    x = a.alloc(1000)            # 1024
    y = a.alloc(2000)            # 2048
    assert a.peak == 3072
    a.free(x)
    z = a.alloc(100)             # 256, in x's place
    assert z == 0 and a.bytes_used == 2304 and a.peak == 3072
    a.alloc(4096)
    assert a.peak == 2304 + 4096
    a.free(y)
    assert a.peak == 2304 + 4096
