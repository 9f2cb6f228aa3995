"""Learned initial poses: training data from the plain method, training of the proposal
network, and its comparison with the Fibonacci initialisation.

The paper initialises particles on a Fibonacci sphere, finds in its ablation (Section VII,
Fig. 3) that a mixture of Gaussians placed with prior knowledge of the object reaches the
same success rate with fewer particles, and names learned initial poses as future work
(Conclusions).  Here the prior is learned: the plain method (Fibonacci initialisation,
Algorithm 1) is run on procedural objects, the best converged particles of every preshape
become the targets, and the proposal network (include/asicp_proposal.h) learns a mixture of
SE(3) densities per preshape from the object cloud.  At test time it proposes fewer particles
for a shorter run.  Every numeric step runs in the library's kernels; this module moves data
between them.
"""
from __future__ import annotations

import time

import numpy as np

from . import asicp, proposal, synth

P_DEFAULT = 3
FWD_SHAPE = asicp.FWD_SHAPES - 1      # the tensor-core matching shape (fastest on these workloads)


def object_clouds(n: int, m: int, seed: int) -> np.ndarray:
    """n seeded procedural partial views of m points (float32 [n, m, 3])."""
    return np.stack([synth.partial_object(m, seed + 7919 * i).points for i in range(n)]).astype(np.float32)


def _context(preshapes, n_obj, K, k_max, stream, init_radius=0.15, k_stein=None):
    P = len(preshapes)
    k_stein = synth.k_stein_for(k_max) if k_stein is None else k_stein
    cfg = asicp.asicp_config_default(P=P, K=int(np.max(K)), k_max=k_max, k_stein=k_stein,
                                     schedule=0, cuda_stream=stream, n_objects=n_obj, init_radius=init_radius,
                                     fwd_shape=FWD_SHAPE)
    ctx = asicp.asicp_create(cfg)
    asicp.asicp_set_particle_counts(ctx, np.full(n_obj * P, K, np.int32) if np.isscalar(K) else K)
    for p, ps in enumerate(preshapes):
        asicp.asicp_set_gripper_sdf(ctx, p, ps.S, ps.sdf, ps.origin, ps.voxel)
    return ctx


def _ranked(ctx, o, n):
    """All particles of object o ranked by the library (non-colliding first, ascending cost)."""
    th = np.zeros((n, 7), np.float32)
    cost = np.zeros(n, np.float32)
    pre = np.zeros(n, np.int32)
    k = asicp.asicp_best_grasps_at(ctx, o, n, th, cost, pre)
    return th[:k], cost[:k], pre[:k]


def converged_targets(clouds, preshapes, K: int = 256, k_max: int = 100, T: int = 16, batch: int = 16,
                      stream=None):
    """Targets [n, P, T, 7]: per object and preshape the T best final poses of the plain method."""
    n, P = len(clouds), len(preshapes)
    out = np.zeros((n, P, T, 7), np.float32)
    best = np.zeros(n, np.float32)
    for s in range(0, n, batch):
        nb = min(batch, n - s)
        ctx = _context(preshapes, nb, K, k_max, stream)
        try:
            for o in range(nb):
                asicp.asicp_set_object_at(ctx, o, clouds[s + o])
            asicp.asicp_run(ctx)
            for o in range(nb):
                th, cost, pre = _ranked(ctx, o, P * K)
                best[s + o] = cost[0]
                for p in range(P):
                    sel = th[pre == p][:T]
                    out[s + o, p] = sel[np.arange(T) % len(sel)]
        finally:
            asicp.asicp_destroy(ctx)
    return out, best


def train(net: proposal.Proposal, clouds, targets, epochs: int, batch: int, lr: float, seed: int):
    """Adam on mini-batches of objects; returns the mean loss per epoch."""
    g = np.random.default_rng(seed)
    n, T = len(clouds), targets.shape[2]
    hist = []
    for _ in range(epochs):
        order = g.permutation(n)
        tot, cnt = 0.0, 0
        for s in range(0, n - batch + 1, batch):
            idx = order[s:s + batch]
            loss, _ = net.loss_grad(np.ascontiguousarray(clouds[idx]), np.ascontiguousarray(targets[idx]), batch, T)
            net.adam_step(lr)
            tot += loss
            cnt += 1
        hist.append(tot / max(cnt, 1))
    return hist


def run_grasp_sets(clouds, preshapes, K: int, k_max: int, stream, theta0=None, batch: int = 16, k_stein=None):
    """Best final cost per object and device time per grasp set (ms), objects batched.  k_stein:
    SVGD iterations (default: Table I's share of k_max)."""
    import torch
    n, P = len(clouds), len(preshapes)
    best = np.zeros(n, np.float32)
    total_ms = 0.0
    for s in range(0, n, batch):
        nb = min(batch, n - s)
        ctx = _context(preshapes, nb, K, k_max, stream, k_stein=k_stein)
        try:
            for o in range(nb):
                asicp.asicp_set_object_at(ctx, o, clouds[s + o])
            th0 = None if theta0 is None else np.ascontiguousarray(theta0[s:s + nb].reshape(-1, 7))
            asicp.asicp_run(ctx, th0)                 # warm-up: captures the loop
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            asicp.asicp_run(ctx, th0)
            for o in range(nb):
                best[s + o] = _ranked(ctx, o, 1)[1][0]
            total_ms += (time.perf_counter() - t0) * 1e3
        finally:
            asicp.asicp_destroy(ctx)
    return best, total_ms / n


def propose(net: proposal.Proposal, clouds, K: int, seed: int, batch: int = 16):
    """K initial poses per preshape for every cloud ([n, P, K, 7]) and the time per object (ms)."""
    import torch
    n, P = len(clouds), net.P
    g = np.random.default_rng(seed)
    out = np.zeros((n, P, K, 7), np.float32)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s in range(0, n, batch):
        nb = min(batch, n - s)
        o, cen = net.forward(np.ascontiguousarray(clouds[s:s + nb]), nb)
        draws = np.concatenate([g.uniform(0, 1, (nb, P, K, 1)), g.normal(size=(nb, P, K, 7))], -1).astype(np.float32)
        out[s:s + nb] = net.sample(o, cen, nb, K, draws)
    return out, (time.perf_counter() - t0) * 1e3 / n


def compare(net, clouds, preshapes, stream, plain=(256, 100), budgets=((64, 30), (64, 20), (64, 10)), seed: int = 5,
            batch: int = 16):
    """Plain method vs learned initialisation vs Fibonacci at the same (particles, iterations)
    budgets, per object.  The learned poses are refined two ways: with the default schedule
    (Table I's share of SVGD iterations, annealing from gamma = 0, i.e. from pure repulsion) and by
    SGD-ICP alone (k_stein = 0), since the proposals already sit near converged poses and the
    annealed repulsion first spreads them out again; Fibonacci is run both ways as well.  For each
    form, the time to reach equal cost on an object is the time of its cheapest budget whose best
    final cost is within 1 % of the plain method's."""
    Kp, kp = plain
    best_plain, ms_plain = run_grasp_sets(clouds, preshapes, Kp, kp, stream, batch=batch)
    target = 1.01 * best_plain
    res = {"objects": len(clouds),
           "plain": {"particles_per_preshape": Kp, "iterations": kp, "ms_per_grasp_set": ms_plain,
                     "median_best_cost": float(np.median(best_plain))},
           "budgets": []}
    forms = ("learned", "learned_sgd", "fibonacci", "fibonacci_sgd")
    reach_ms = {f: np.full(len(clouds), np.inf) for f in forms}
    for Kl, kl in budgets:
        th0, ms_prop = propose(net, clouds, Kl, seed, batch=batch)
        out = {
            "learned": run_grasp_sets(clouds, preshapes, Kl, kl, stream, theta0=th0, batch=batch),
            "learned_sgd": run_grasp_sets(clouds, preshapes, Kl, kl, stream, theta0=th0, batch=batch, k_stein=0),
            "fibonacci": run_grasp_sets(clouds, preshapes, Kl, kl, stream, batch=batch),
            "fibonacci_sgd": run_grasp_sets(clouds, preshapes, Kl, kl, stream, batch=batch, k_stein=0)}
        entry = {"particles_per_preshape": Kl, "iterations": kl, "proposal_ms": ms_prop,
                 "ms_per_grasp_set": {}, "reach_plain_cost_within_1pct": {}, "median_cost_ratio_vs_plain": {}}
        for f in forms:
            best, ms = out[f]
            ms = ms + (ms_prop if f.startswith("learned") else 0.0)
            ok = best <= target
            reach_ms[f] = np.where(ok, np.minimum(reach_ms[f], ms), reach_ms[f])
            entry["ms_per_grasp_set"][f] = ms
            entry["reach_plain_cost_within_1pct"][f] = float(np.mean(ok))
            entry["median_cost_ratio_vs_plain"][f] = float(np.median(best / np.maximum(best_plain, 1e-30)))
        entry["learned_sgd_beats_fibonacci"] = float(np.mean(out["learned_sgd"][0] < out["fibonacci"][0]))
        entry["learned_sgd_beats_fibonacci_sgd"] = float(np.mean(out["learned_sgd"][0] < out["fibonacci_sgd"][0]))
        res["budgets"].append(entry)
    res["equal_cost"] = {}
    for f in forms:
        r = np.isfinite(reach_ms[f])
        res["equal_cost"][f] = {
            "objects_reaching": float(np.mean(r)),
            "median_ms_when_reached": float(np.median(reach_ms[f][r])) if r.any() else None,
            "median_speedup_vs_plain_when_reached": float(np.median(ms_plain / reach_ms[f][r])) if r.any() else None}
    return res
