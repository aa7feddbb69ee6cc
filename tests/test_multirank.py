"""The N-rank bench aggregation on CPU with gloo, world size 2: each rank
resamples its own image (replicas, no data-path collective); the job time is
the slowest rank's, the throughput counts every rank's pixels."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_s = [2.0, 3.0][rank]
    value, job_s = bench.aggregate(units_per_step=1000, steps=10, local_seconds=local_s, world=world)
    bench.barrier(world)
    q.put((rank, value, job_s))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, job_s in res:
        assert job_s == 3.0                       # the slowest rank sets the job time
        assert value == pytest.approx(1000 * 10 * 2 / 3.0)


def test_single_rank_aggregation():
    import bench
    value, job_s = bench.aggregate(500, 4, 2.0, 1)
    assert (value, job_s) == (1000.0, 2.0)
