"""bench.py --gpus N runs N independent replicas of the workload (the path has
no exchange step on one GPU): the job's time is the slowest rank's and its
throughput counts every replica.  Checked with two gloo ranks on the CPU."""

import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")
    dist.barrier()
    out.put((rank, t, bench.job_value(world, 100, 7, t)))
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_sum_the_work():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [2.0, 2.0]
    assert res[0][2] == pytest.approx(2 * 100 * 7 / 2.0)


def test_without_process_group_the_value_is_the_local_one():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_value(1, 10, 3, 2.0) == 15.0
