"""Host-side sharding of AS-ICP work over several GPUs (one process per GPU).

The method partitions cleanly: objects are independent problems, and the
preshapes of one object couple only through the final choice of the best grasp
(Stein updates act within a preshape; Algorithm 1's argmin is over all
particles).  So a grasp set can be split by preshape across ranks, each rank
running the whole iteration loop on its preshapes with no exchange, followed by
one merge of the per-rank top-k lists; many objects are split by object with
no exchange at all.  The merge uses the same ranking as the library:
non-colliding first, ascending cost, ties to the lower global (preshape, particle)
index.
"""
from __future__ import annotations

import numpy as np


def shard(n_items: int, world: int, rank: int) -> list[int]:
    """Contiguous block of item indices for `rank` (sizes differ by at most one)."""
    base, extra = divmod(n_items, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))


def rank_key(colliding: np.ndarray, cost: np.ndarray, global_index: np.ndarray) -> np.ndarray:
    """Sort order of candidate grasps: non-colliding, then cost (NaN last), then index."""
    c = np.where(np.isnan(cost), np.inf, cost)
    return np.lexsort((global_index, c, colliding.astype(np.int8)))


def merge_topk(parts: list[dict], topk: int) -> dict:
    """Merge per-rank candidate lists.  Each part holds arrays 'theta' (n, 7),
    'cost' (n,), 'colliding' (n,), 'index' (n,) where index is the global flat
    particle index preshape * K + j."""
    theta = np.concatenate([p["theta"] for p in parts]) if parts else np.zeros((0, 7), np.float32)
    cost = np.concatenate([p["cost"] for p in parts]) if parts else np.zeros(0)
    col = np.concatenate([p["colliding"] for p in parts]) if parts else np.zeros(0, bool)
    idx = np.concatenate([p["index"] for p in parts]) if parts else np.zeros(0, np.int64)
    order = rank_key(col, cost, idx)[:topk]
    return {"theta": theta[order], "cost": cost[order], "colliding": col[order], "index": idx[order]}


def gather_merge_topk(local: dict, topk: int, group=None) -> dict:
    """All ranks contribute their candidate list; every rank receives the merged top-k
    (torch.distributed, any backend that supports object collectives)."""
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [None] * world
    dist.all_gather_object(parts, {k: np.asarray(v) for k, v in local.items()}, group=group)
    return merge_topk(parts, topk)


def max_over_ranks(value: float, group=None) -> float:
    """Largest value over all ranks (the step time of a weak-scaling run)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
