"""The multi-process path of bench.py (replicas, slowest-rank time, whole-job throughput) on CPU with gloo."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def worker(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, dist, "cpu")
    v = bench.job_throughput(world, 131072, 4000, 3, t)
    dist.barrier()
    q.put((rank, t, v))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time, and the whole-job value counts both replicas
    assert res[0][1] == res[1][1] == 2.5
    assert res[0][2] == pytest.approx(2 * 131072 * 4000 * 3 / 2.5 / 1e9)


def test_single_process_identity():
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    assert bench.max_over_ranks(3.25, None, "cpu") == 3.25


def shard_worker(rank, world, port, q):
    import sys

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import numpy as np

    import bench
    from paper_2608_01071_b300.workloads import batched_study

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    sizes = [int(np.prod(w["shape"])) for w in batched_study()]
    mine = bench.shard_instances(sizes, rank, world)
    got = [None] * world
    dist.all_gather_object(got, mine)
    q.put((rank, got, sizes))
    dist.destroy_process_group()


def test_two_rank_instance_sharding_gloo():
    # the batched study split over two ranks: every rank derives the same partition, shards are disjoint, cover
    # all instances, and their node counts differ by at most one instance's size
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=shard_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, got0, sizes), (_, got1, _) = res
    assert got0 == got1
    a, b = got0
    assert not set(a) & set(b) and sorted(a + b) == list(range(len(sizes)))
    la, lb = sum(sizes[i] for i in a), sum(sizes[i] for i in b)
    assert abs(la - lb) <= max(sizes)
