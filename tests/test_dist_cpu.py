"""The multi-rank host path of bench.py on CPU (gloo, world size 2): the instance shards
cover every game exactly once, the timing reduction takes the maximum over ranks, and the
per-rank result lists are gathered. The data path itself has no collective."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = list(bench.shard(1024, rank, world))
    got = bench.gather_lists([float(v) for v in mine], world)
    t = bench.max_over_ranks(1.0 + rank, world)
    bench.barrier(world)
    q.put((rank, len(mine), sorted(int(v) for v in got), t))
    dist.destroy_process_group()


def test_shards_cover_all_instances_once():
    sys.path.insert(0, ROOT)
    import bench
    for count in (1, 7, 1024, 1025):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                seen += list(bench.shard(count, r, world))
            assert sorted(seen) == list(range(count))


def test_gloo_two_ranks():
    import multiprocessing as mp
    import socket
    ctx = mp.get_context("spawn")
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, n_mine, got, t in out:
        assert n_mine == 512
        assert got == list(range(1024))
        assert t == 2.0
