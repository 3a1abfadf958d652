"""Continuous batching: each served result equals the frame's result run
alone, with several batches in flight, under an HBM admission budget, and in
the plain per-frame mode."""
import numpy as np
import pytest

from paper_2003_11076_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pool():
    from paper_2003_11076_gb300 import build
    build.build()
    frames = [scenes.small_gray(i, H=40 + 7 * i, W=64 + 13 * i, M=15, D=16 + 4 * (i % 3), iters=3 + i % 4)
              for i in range(6)]
    frames += [scenes.small_gray(20, baselines=[-0.3, -0.1, 0.0, 0.2, 0.35, 0.5, 0.6], D=24, iters=5),
               scenes.street_rgb(1, H=64, W=96, D=32, iters=6, M=30),
               scenes.random_frame(1, scale=0.2)]
    return frames


def _check_equal_alone(lf, reqs, frames):
    for r in reqs:
        alone = lf.run_scene(frames[r.rid % len(frames)])
        g = r.result
        assert np.array_equal(g["d_idx"], alone["d_idx"])
        assert np.array_equal(g["labels"].view(np.uint16), alone["labels"])
        assert np.max(np.abs(g["post"] - alone["post"])) <= 1e-6
        assert np.max(np.abs(g["refocus"] - alone["refocus"])) <= 1e-6


def test_served_results_equal_alone_with_batches_in_flight(pool):
    from paper_2003_11076_gb300 import lf, serve
    srv = serve.Server(max_batch=3, inflight=2)
    reqs = [serve.Request.from_scene(i, pool[i % len(pool)], arrival=0.002 * i) for i in range(18)]
    rep = srv.run_arrivals(reqs)
    assert rep["requests"] == 18 and rep["batches"] >= 6
    _check_equal_alone(lf, srv.completed, pool)
    srv.close()


def test_admission_respects_hbm_budget(pool):
    from paper_2003_11076_gb300 import lf, serve
    reqs = [serve.Request.from_scene(i, pool[i % len(pool)]) for i in range(9)]
    biggest = max(r.device_bytes() for r in reqs)
    srv = serve.Server(max_batch=8, inflight=2, hbm_budget=2 * biggest)
    for r in reqs:
        srv.submit(r)
    srv.drain()
    assert len(srv.completed) == 9
    assert srv.peak_admitted <= 2 * biggest // min(r.device_bytes() for r in reqs)
    assert srv.admitted_bytes == 0
    _check_equal_alone(lf, srv.completed, pool)
    srv.close()


def test_plain_per_frame_mode(pool):
    from paper_2003_11076_gb300 import lf, serve
    srv = serve.Server(mode="plain")
    reqs = [serve.Request.from_scene(i, pool[i % len(pool)], arrival=0.0) for i in range(len(pool))]
    rep = srv.run_arrivals(reqs)
    assert rep["requests"] == len(pool)
    _check_equal_alone(lf, srv.completed, pool)


def test_reduced_precision_served_equals_alone(pool):
    from paper_2003_11076_gb300 import lf, serve
    p = lf.default_params(precision=1)
    srv = serve.Server(p, max_batch=4, inflight=2)
    reqs = [serve.Request.from_scene(i, pool[i % len(pool)], arrival=0.0) for i in range(8)]
    srv.run_arrivals(reqs)
    for r in srv.completed:
        alone = lf.run_scene(pool[r.rid % len(pool)], params=lf.default_params(precision=1))
        assert np.array_equal(r.result["d_idx"], alone["d_idx"])
    srv.close()
