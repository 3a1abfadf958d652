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


def test_request_larger_than_the_budget_is_rejected_not_left_waiting(pool):
    """A frame whose buffers exceed the server's whole device block can never
    be admitted: submit rejects it at once (status and message), and the
    other requests are served normally."""
    from paper_2003_11076_gb300 import lf, serve
    small = [serve.Request.from_scene(i, pool[i]) for i in range(3)]
    big = serve.Request.from_scene(99, scenes.street_rgb(0, H=400, W=640, D=32, iters=3, M=40))
    budget = max(r.device_bytes() for r in small) * 2
    assert big.device_bytes() > budget
    srv = serve.Server(max_batch=4, inflight=2, hbm_budget=budget)
    assert not srv.submit(big)
    assert big.status == "rejected" and "device bytes" in big.error
    for r in small:
        assert srv.submit(r)
    srv.drain(timeout_s=60)
    assert [r.status for r in small] == ["done"] * 3 and srv.rejected == [big]
    assert srv.admitted_bytes == 0
    _check_equal_alone(lf, small, pool)
    srv.close()


def test_cancelled_requests_return_their_bytes(pool):
    """Cancelling a request that waits for admission, or one admitted but not
    launched, returns its device and host bytes; a launched one cannot be
    cancelled; the rest complete with their results."""
    from paper_2003_11076_gb300 import lf, serve
    reqs = [serve.Request.from_scene(i, pool[i]) for i in range(4)]
    srv = serve.Server(max_batch=4, inflight=1, hbm_budget=sum(r.device_bytes() for r in reqs))
    for r in reqs:
        srv.submit(r)
    assert srv.cancel(reqs[3]) and reqs[3].status == "cancelled"   # still pending
    srv._admit()                                                     # admitted, not launched
    used = srv.admitted_bytes
    assert reqs[2].status == "admitted" and srv.cancel(reqs[2])
    assert srv.admitted_bytes < used and reqs[2].status == "cancelled"
    srv._launch()
    assert not srv.cancel(reqs[0])                                   # on the GPU
    srv.drain(timeout_s=60)
    assert [r.status for r in reqs] == ["done", "done", "cancelled", "cancelled"]
    assert srv.admitted_bytes == 0 and srv.dev_arena.free_list == [(0, srv.dev_arena.capacity)]
    _check_equal_alone(lf, reqs[:2], pool)
    srv.close()
