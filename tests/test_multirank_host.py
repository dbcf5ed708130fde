"""The multi-rank host path of the benchmark on CPU: two gloo ranks, each
with its own replica's timing, agree on the slowest rank's time and report
the whole job's throughput (queries of all ranks / that time)."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r took (r + 1) * 100 ms for 10 steps of 1000 queries
    ms, value = bench.aggregate_timing(100.0 * (rank + 1), 10, 1000, world, "cpu")
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, value in got:
        assert ms == pytest.approx(20.0)                  # 200 ms / 10 steps, the slower rank
        assert value == pytest.approx(2 * 1000 / 0.020)   # both ranks' queries per second


def test_single_rank_needs_no_process_group():
    import bench
    ms, value = bench.aggregate_timing(50.0, 5, 200, 1, "cpu")
    assert ms == 10.0 and value == pytest.approx(200 / 0.010)
