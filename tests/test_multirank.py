"""The multi-GPU path's host logic on CPU: two gloo ranks shard a batch of
views with no data collective (the shards partition the views, balanced by
point count), derive distinct per-rank frame seeds for weak scaling, and
agree on the max-over-ranks step time the benchmark reports."""
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2508_19140_gb300 import scenes
from paper_2508_19140_gb300.shard import rank_seed, shard_views


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            init_method=f"tcp://127.0.0.1:{port}")
    counts = [n for (_, _, n) in scenes.BATCH_VIEWS]
    mine = shard_views(counts, world, rank)
    shards = [None] * world
    dist.all_gather_object(shards, mine)
    t = torch.tensor([1.5 * (rank + 1)], dtype=torch.float64)  # a rank's step time
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    seeds = [None] * world
    dist.all_gather_object(seeds, rank_seed(2, rank))
    dist.barrier()
    q.put((rank, shards, float(t.item()), seeds))
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_views_and_reduce_time():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    counts = [n for (_, _, n) in scenes.BATCH_VIEWS]
    for rank, shards, tmax, seeds in out:
        flat = sorted(k for s in shards for k in s)
        assert flat == list(range(len(counts)))           # a partition of the views
        loads = [sum(counts[k] for k in s) for s in shards]
        assert max(loads) - min(loads) <= max(counts)      # greedy balance bound
        assert tmax == 3.0                                 # max over ranks
        assert len(set(seeds)) == world                    # independent frames


def test_shard_views_edge_cases():
    assert shard_views([5], 1, 0) == [0]
    assert shard_views([], 3, 1) == []
    assert shard_views([1, 1, 1, 1], 4, 2) == [2]
    with pytest.raises(ValueError):
        shard_views([1], 2, 2)
