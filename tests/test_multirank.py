"""The benchmark's multi-rank (replicas) bookkeeping on two gloo ranks (CPU):
the timed region is the slowest rank's, the value all ranks' work over it."""
import multiprocessing as mp
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    w, r, loc = bench.dist_setup()
    t = bench.max_over_ranks(1.5 + rank)            # rank 1 is the slower one
    v = bench.whole_job_value(units_per_rank=300.0, world=w, seconds=t)
    dist.barrier()
    q.put((r, w, t, v))
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_weak_scaling_value():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, (r, w, t, v) in enumerate(got):
        assert (r, w) == (rank, 2)
        assert t == pytest.approx(2.5)                # max over ranks
        assert v == pytest.approx(300.0 * 2 / 2.5)    # all ranks' units / slowest time


def test_single_process_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25
    assert bench.whole_job_value(10.0, 1, 2.0) == 5.0
