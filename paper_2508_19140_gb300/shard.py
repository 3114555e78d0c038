"""Host-side partitioning of rasterization work across GPUs.

Views are independent problems (each view has its own point cloud in the
paper's view-specific sampling, Sec. 2 "Point Cloud Sampling"), so several
GPUs split them with no collective on the data path: each rank rasterizes
its own views, and only timing needs a reduction. Weak scaling gives every
rank a whole frame of its own (its own seed); strong scaling splits one
batch of views by point count.
"""
from __future__ import annotations


def rank_seed(config_id: int, rank: int) -> int:
    """Seed of the frame rank `rank` renders under weak scaling."""
    return 1000 + config_id + 7919 * rank


def shard_views(point_counts, world: int, rank: int) -> list:
    """Balanced, deterministic split of views over ranks: views in descending
    point count go to the currently least-loaded rank (lowest rank on ties).
    Returns the sorted view indices of `rank`; the shards partition the views."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    load = [0] * world
    owner = {}
    order = sorted(range(len(point_counts)), key=lambda k: (-int(point_counts[k]), k))
    for k in order:
        r = min(range(world), key=lambda q: (load[q], q))
        owner[k] = r
        load[r] += int(point_counts[k])
    return sorted(k for k, r in owner.items() if r == rank)
