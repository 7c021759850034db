"""The multi-GPU bench path runs independent replicas (no data-path collective); only the timing
is combined: the job's time is the slowest rank's and the value counts every rank's work.
Exercised here with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [40.0, 55.0][rank]                      # per-rank step times
    worst = bench.max_over_ranks(ms, dist, "cpu")
    value = bench.job_rate(1.0e12, world, worst * 1e-3)
    q.put((rank, worst, value))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    for rank, worst, value in res:
        assert worst == 55.0
        assert value == pytest.approx(2 * 1.0e12 / 0.055)
