"""The N > 1 path on CPU: two gloo ranks, each with its own shard (weak
scaling); the job time is the slowest rank's and the throughput counts the
units of every rank.  No collective touches the data: only the elapsed time
is reduced.  The sharding itself (element ranges, the node subset of an
indexed shard) is checked by running the oracle per rank on its shard: the
outputs concatenated in rank order equal one rank's on the whole mesh."""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
import oracle
from paper_1706_01613_gb300 import shard, synth


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


def _shard_rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    nodes, conn = synth.structured_grid(13, 11, 9, sigma=0.3, seed=611)
    n_nodes, n_conn, (lo, hi), ids = shard.shard_indexed(nodes, conn, rank, world)
    f, bmin, bmax = oracle.check_indexed(n_nodes, n_conn, max_depth=8, threads=1)
    X = synth.twisted_layers(3001, seed=612, theta_max_deg=150.0)
    xs, (slo, shi) = shard.shard_soa(X, rank, world)
    fs, _, _ = oracle.check_soa(xs, max_depth=8, threads=1)
    # the test collects the per-rank outputs to compare them; the data path
    # itself exchanges nothing
    parts = [None] * world
    dist.all_gather_object(parts, (rank, lo, hi, f, bmin, bmax, len(ids), slo, shi, fs))
    if rank == 0:
        q.put(parts)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_of_one_mesh_concatenate_to_the_single_rank_result():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_shard_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    parts = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts.sort(key=lambda t: t[0])
    nodes, conn = synth.structured_grid(13, 11, 9, sigma=0.3, seed=611)
    want = oracle.check_indexed(nodes, conn, max_depth=8)
    assert [p[1] for p in parts] == [0, parts[0][2]] and parts[-1][2] == len(conn)
    assert all(p[6] < nodes.shape[0] for p in parts)  # each rank holds a node subset
    for k in (3, 4, 5):
        assert np.array_equal(np.concatenate([p[k] for p in parts]), want[k - 3])
    X = synth.twisted_layers(3001, seed=612, theta_max_deg=150.0)
    wf, _, _ = oracle.check_soa(X, max_depth=8)
    assert np.array_equal(np.concatenate([p[9] for p in parts]), wf)
    assert (wf >> 3 & 15).max() >= 1  # refinement happens inside the shards


def test_element_ranges_and_renumbering():
    for n, world in ((10, 3), (0, 2), (7, 7), (5, 8)):
        r = [shard.element_range(n, k, world) for k in range(world)]
        assert r[0][0] == 0 and r[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(r, r[1:]))
        assert max(h - l for l, h in r) - min(h - l for l, h in r) <= 1
    nodes, conn = synth.structured_grid(6, 5, 4, sigma=0.2, seed=613)
    conn = conn.copy()
    conn[7, 3] = -1
    conn[30, 0] = nodes.shape[0]
    for world in (1, 2, 3):
        rows = []
        for rank in range(world):
            ln, lc, (lo, hi), ids = shard.shard_indexed(nodes, conn, rank, world)
            assert np.all(np.diff(ids) > 0) and np.array_equal(ln, nodes[ids])
            ok = (lc < len(ids))
            glob = np.where(ok, ids[np.minimum(lc, len(ids) - 1)], -1)
            want = np.where((conn[lo:hi] >= 0) & (conn[lo:hi] < nodes.shape[0]), conn[lo:hi], -1)
            assert np.array_equal(glob, want)
            rows.append(lc)
        assert sum(len(r) for r in rows) == len(conn)
