"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own
shard (weak scaling); the job time is the slowest rank's and the
throughput counts the units of every rank.  No collective touches the data:
only the elapsed time is reduced."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)  # rank 1 is slower
    value, total = bench.aggregate(local_ms, 1000, 10, world, dist)
    dist.barrier()
    q.put((rank, value, total))
    dist.destroy_process_group()


def test_two_ranks_weak_scaling_uses_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, value, total in out:
        assert total == pytest.approx(200.0)
        assert value == pytest.approx(2 * 1000 * 10 / 0.2)


def test_single_rank_needs_no_collective():
    value, total = bench.aggregate(50.0, 100, 4, 1)
    assert total == 50.0 and value == pytest.approx(100 * 4 / 0.05)
