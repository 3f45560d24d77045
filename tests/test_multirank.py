"""bench.py's multi-process host logic on CPU: two gloo ranks (replicas)."""
import os

import pytest
import torch.multiprocessing as mp


def _rank(rank, world, port, q):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo")
    bench.barrier(world)
    local_ms = 100.0 * (rank + 1)                 # rank 1 is the slow replica
    value, t = bench.whole_job_rate(200, local_ms, world)
    q.put((rank, value, t))
    dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_time_and_the_whole_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29617
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, t in res:
        assert t == pytest.approx(200.0)           # max over ranks
        assert value == pytest.approx(2 * 200 / 0.2)   # all ranks' units / slowest time


def test_single_rank_needs_no_process_group():
    import bench
    value, t = bench.whole_job_rate(20, 10.0, 1)
    assert t == 10.0 and value == pytest.approx(2000.0)
