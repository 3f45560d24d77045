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


def test_dominant_phase_counts_every_launch_of_a_phase():
    """The dominant kernel class is chosen by its time per PD iteration: a
    phase split over two launches counts both; near-ties go to the larger
    byte stream; the kernels outside the iteration loop are not candidates."""
    import bench
    times = {"dd_interior": 0.030, "dd_condense": 0.026, "local": 0.031, "inertia": 0.5, "velocity": 0.4}
    nbytes = {"dd_interior": 71_000_000, "dd_condense": 48_000_000, "local": 44_000_000}
    assert bench.dominant_phase(times, nbytes, {"dd_interior": 2, "dd_condense": 1, "local": 1}) == "dd_interior"
    assert bench.dominant_phase(times, nbytes, {"dd_interior": 1, "dd_condense": 1, "local": 1}) == "dd_interior"
    assert bench.dominant_phase({"local": 0.031, "dd_condense": 0.020}, nbytes, {}) == "local"


def test_clock_samples_are_read_inside_the_timed_window(tmp_path):
    """nvidia-smi samples outside the timed window do not count; a throttle
    reason active inside it is reported (such a run is re-measured)."""
    import datetime
    import bench
    t0 = datetime.datetime(2026, 1, 1, 12, 0, 0).timestamp()
    rows = []
    for k, (mhz, hw) in enumerate([(1200.0, "Not Active"), (2070.0, "Not Active"), (2070.0, "Active"),
                                   (2055.0, "Not Active"), (900.0, "Not Active")]):
        ts = datetime.datetime.fromtimestamp(t0 + 0.3 * k).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        rows.append(f"{ts}, 0, {mhz}, 2070, 900.0, 0x0, {hw}, Not Active, Not Active, Not Active")
    p = tmp_path / "clocks.csv"
    p.write_text("\n".join(rows) + "\n")
    out = bench.ClockSampler.summarize(str(p), t0 + 0.25, t0 + 0.95)   # samples 1, 2, 3
    assert out["samples"] == 3 and out["in_timed_window"]
    assert out["sm_mhz"] == 2070.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["hw_slowdown"]
    everything = bench.ClockSampler.summarize(str(p), None, None)
    assert everything["samples"] == 5 and not everything["in_timed_window"]
