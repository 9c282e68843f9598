"""Host logic of the multi-GPU benchmark path on CPU: two ranks joined over gloo (world size 2).

Instances are independent solves, so the N-GPU bench shards them across ranks with no collective on the
data path; the only collectives are a barrier and the maximum of the ranks' timings.  These tests run
that logic with the gloo backend: the shards of all ranks are disjoint and cover the seeded stream, the
timing reduction returns the slowest rank, and the reference arm does its work on rank 0 only.
"""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WORLD = 2
N_SETS, B = 5, 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, port, q):
    try:
        os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(WORLD), RANK=str(rank),
                          LOCAL_RANK=str(rank))
        sys.path.insert(0, ROOT)
        import torch
        import torch.distributed as dist
        import bench
        world, r, _ = bench.dist_setup("gloo")
        assert (world, r) == (WORLD, rank)
        mine = [bench.shard(r, N_SETS, B, step) for step in range(N_SETS)]
        gathered = [None] * world
        dist.all_gather_object(gathered, mine)
        bench.barrier(world)
        slowest = bench.max_over_ranks(world, 1.5 + r)
        # the reference arm: rank 0 alone works, the other ranks return at once
        class Args:
            steps, warmup, ref_iters, ref_cores, workload, restart, rom_rank = 1, 1, 10.0, 1, "slab1d_128", 30, 0
        called = []
        orig = bench.oracle_baseline
        bench.oracle_baseline = lambda *a, **k: called.append(1) or {"value": 1.0, "cores": 1, "sample": "x",
                                                                     "per_iter_samples": [0.1]}
        bench.run_reference(Args, bench.wl.config(1), 1, world, r, 1)
        bench.oracle_baseline = orig
        dist.destroy_process_group()
        q.put((rank, gathered, slowest, len(called)))
    except BaseException as e:   # report instead of hanging the parent
        q.put((rank, repr(e), None, None))


def test_two_ranks_shard_disjointly_and_reduce_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    results = {}
    for _ in range(WORLD):
        rank, gathered, slowest, ncalls = q.get(timeout=240)
        results[rank] = (gathered, slowest, ncalls)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in range(WORLD):
        gathered, slowest, ncalls = results[rank]
        assert not isinstance(gathered, str), gathered
        assert slowest == 1.5 + (WORLD - 1)
        if rank > 0:
            assert ncalls == 0
        else:
            assert ncalls >= 1
    gathered = results[0][0]
    draws = sorted(i for shards in gathered for (i0, i1) in shards for i in range(i0, i1))
    assert draws == list(range(WORLD * N_SETS * B))       # disjoint and covering
    assert gathered == results[1][0]
