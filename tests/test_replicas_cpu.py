"""The multi-GPU path is replicas only (views are independent; nothing is exchanged inside a
frame). Its host logic -- which views a replica renders and the job time as the slowest
replica's -- runs here as two gloo ranks on the CPU."""
import os
import socket

import pytest


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
    steps = 5
    first = bench.replica_first_view(rank, steps)
    views = [(first + i) % 32 for i in range(steps)]
    t = bench.max_over_ranks(1.0 + rank, dist, "cpu")   # replica r took 1 + r ms
    q.put((rank, views, t))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_shard_views_and_take_the_slowest_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    (_, v0, t0), (_, v1, t1) = out
    assert set(v0).isdisjoint(v1) and len(v0) == len(v1) == 5
    assert t0 == t1 == 2.0


def test_one_rank_keeps_its_own_time():
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.replica_first_view(0, 32) == 0
