"""Multi-rank host logic on CPU with the gloo backend (world size 2): sharding by
preshape followed by the final top-k merge gives the same ranking as one process
that ranks every particle, and the step time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2412_08346_gb300 import dist as adist  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(P=5, K=7, seed=3):
    g = np.random.default_rng(seed)
    cost = g.uniform(0, 1e-3, (P, K))
    cost[1, 2] = cost[3, 4]                       # a tie across preshapes (and ranks)
    col = g.uniform(0, 1, (P, K)) < 0.25
    theta = g.normal(size=(P, K, 7)).astype(np.float32)
    return cost, col, theta


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cost, col, theta = _problem()
        P, K = cost.shape
        mine = adist.shard(P, world, rank)
        local = {"theta": theta[mine].reshape(-1, 7), "cost": cost[mine].ravel(),
                 "colliding": col[mine].ravel(),
                 "index": np.array([p * K + j for p in mine for j in range(K)], np.int64)}
        merged = adist.gather_merge_topk(local, topk=10)
        tmax = adist.max_over_ranks(1.0 + rank)
        out[rank] = (merged["index"].tolist(), tmax, mine)
    finally:
        dist.destroy_process_group()


def test_preshape_sharding_and_topk_merge_match_single_process():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    cost, col, theta = _problem()
    P, K = cost.shape
    ref = adist.rank_key(col.ravel(), cost.ravel(), np.arange(P * K))[:10].tolist()
    import oracle
    assert ref == oracle.select(cost.ravel(), col.ravel().astype(np.int32), 10).tolist()
    for r in range(world):
        idx, tmax, mine = out[r]
        assert idx == ref
        assert tmax == 2.0
    assert sorted(out[0][2] + out[1][2]) == list(range(P))


def test_shard_sizes():
    for n in (1, 3, 7, 64):
        for world in (1, 2, 3, 8):
            parts = [adist.shard(n, world, r) for r in range(world)]
            assert sum(parts, []) == list(range(n))
            assert max(map(len, parts)) - min(map(len, parts)) <= 1
