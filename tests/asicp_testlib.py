"""Helpers shared by the parity tests: set a workload up on both sides and
compare the CUDA path (through the C-ABI binding) with the FP64 oracle.

Tolerances:
* correspondences: bit-exact, except near-ties where the FP64 squared distance
  of the GPU's choice exceeds the minimum by at most NEAR_TIE_REL relative (the
  float32 exact-form distance the GPU ranks by has ~3 ulp = 2e-7 relative error);
* collision flags: equal, except points whose FP64 SDF value lies within
  PHI_TOL of zero (float32 transform and interpolation error is ~1e-7 m);
* cost and gradient: relative error <= COST_GRAD_REL per particle and per block
  (translation, quaternion) when both are evaluated on the same pairs.
"""
from __future__ import annotations

import numpy as np

from paper_2412_08346_gb300 import asicp, synth

NEAR_TIE_REL = 1e-6
PHI_TOL = 1e-6
COST_GRAD_REL = 1e-4
# absolute floors for values at the rounding level of the per-particle sums (a cost
# or gradient that cancels to ~0 has no meaningful relative error): the sums carry
# ~1e-14 relative error of terms of magnitude <= ~0.1 m^2 / 0.3 m
COST_ABS = 1e-14
GRAD_ABS = 1e-13


def make_config(w: synth.Workload, stream=None, debug=True, profile=False, **over):
    cfg = asicp.asicp_config_default(P=len(w.preshapes), K=w.K, k_max=w.k_max, k_stein=w.k_stein,
                                     schedule=w.schedule, g0=w.g0, g1=w.g1, C_cycles=w.C_cycles, p_exp=w.p_exp,
                                     conv_tol=-1.0, debug=int(debug), profile=int(profile))
    if stream is not None:
        cfg.cuda_stream = stream
    for k, v in over.items():
        setattr(cfg, k, v)
    return cfg


def upload(ctx, w: synth.Workload, obj_index=0, device=True):
    """Set object and preshapes; device=True passes CUDA tensors, else host numpy arrays."""
    import torch
    obj = w.objects[obj_index].points

    def arr(x):
        x = np.ascontiguousarray(x)
        return torch.from_numpy(x).cuda() if device else x
    keep = []
    R = arr(obj)
    keep.append(R)
    asicp.asicp_set_object(ctx, R)
    for p, pre in enumerate(w.preshapes):
        S, g = arr(pre.S), arr(pre.sdf)
        keep += [S, g]
        asicp.asicp_set_gripper_sdf(ctx, p, S, g, pre.origin, pre.voxel)
    if device:
        torch.cuda.synchronize()
    return keep


def make_oracle(w: synth.Workload, obj_index=0):
    import oracle
    return oracle.Oracle(np.stack([pre.S for pre in w.preshapes]),
                         [(pre.sdf, pre.origin, pre.voxel) for pre in w.preshapes],
                         w.objects[obj_index].points, K=w.K)


def read_state(ctx, P, K, N, Mc, debug=True):
    PK = P * K
    st = {"theta": np.zeros((PK, 7), np.float32), "cost": np.zeros(PK), "grad": np.zeros((PK, 7)),
          "phi": np.zeros((PK, 7), np.float32), "ncol": np.zeros(PK, np.int32), "frozen": np.zeros(PK, np.int32),
          "h": np.zeros(P, np.float32)}
    if debug:
        st.update({"nn_idx": np.zeros((PK, N), np.int32), "nn_d2": np.zeros((PK, N), np.float32),
                   "s_prime": np.zeros((PK, N, 3), np.float32), "col_list": np.zeros((PK, Mc), np.int32),
                   "col_nn": np.zeros((PK, Mc), np.int32)})
    asicp.asicp_get_state(ctx, **st)
    return st


def read_theta(ctx, PK):
    th = np.zeros((PK, 7), np.float32)
    asicp.asicp_get_state(ctx, theta=th)
    return th


def check_nn(queries32, refs32, idx_gpu, report, kind="nn"):
    """Correspondences against the FP64 argmin over the GPU's own float32 queries."""
    import oracle
    q = np.asarray(queries32, np.float64).reshape(-1, 3)
    r = np.asarray(refs32, np.float64).reshape(-1, 3)
    idx_o, d2_o = oracle.nn(q, r)
    g = np.asarray(idx_gpu).reshape(-1)
    mism = np.nonzero(g != idx_o)[0]
    report[f"{kind}_total"] = report.get(f"{kind}_total", 0) + len(g)
    if len(mism):
        d2_g = ((q[mism] - r[g[mism]]) ** 2).sum(1)
        ok = d2_g - d2_o[mism] <= NEAR_TIE_REL * d2_o[mism]
        report[f"{kind}_near_ties"] = report.get(f"{kind}_near_ties", 0) + int(ok.sum())
        bad = mism[~ok]
        assert len(bad) == 0, (f"{len(bad)} correspondences differ beyond a near-tie, e.g. query {bad[0]}: gpu "
                               f"{g[bad[0]]} d2={((q[bad[0]] - r[g[bad[0]]]) ** 2).sum():.9e} vs oracle "
                               f"{idx_o[bad[0]]} d2={d2_o[bad[0]]:.9e}")
    return idx_o


def rel_err(a, b, floor=0.0):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), floor)


def check_step(orc, w, before_theta, st, k, report, check_update=True, sample=None, prior=None):
    """Teacher-forced comparison of one GPU step against the oracle, particle by particle.
    prior: None or (sigma_t, kappa_q, mean_q, CoM) of the Stein direction's priors."""
    import oracle
    P, K, N = orc.P, orc.K, orc.N
    Mc = len(orc.Cc)
    pks = range(P * K) if sample is None else sample
    flips = set()
    for pk in pks:
        p = pk // K
        th = before_theta[pk].astype(np.float64)
        # forward pairs: exact or near-tie against FP64 argmin over the GPU's s'
        check_nn(st["s_prime"][pk], orc.R, st["nn_idx"][pk], report)
        # collision flags
        lst_o, vals = orc.collision_points(p, th)
        n_g = int(st["ncol"][pk])
        lst_g = st["col_list"][pk, :n_g]
        if not np.array_equal(lst_g, lst_o):
            diff = np.setxor1d(lst_g, lst_o)
            assert np.all(np.abs(vals[diff]) <= PHI_TOL), f"particle {pk}: collision flags differ beyond |phi| <= {PHI_TOL}"
            flips.add(pk)
            report["col_flips"] = report.get("col_flips", 0) + len(diff)
            continue
        report["col_points"] = report.get("col_points", 0) + n_g
        if n_g > 0:
            Cc = orc.Cc
            check_nn(Cc[lst_g], st["s_prime"][pk], st["col_nn"][pk, :n_g], report, kind="col_nn")
            cost_o, g_o = orc.collision_terms(p, th, lst_g, st["col_nn"][pk, :n_g])
            report["colliding_particles"] = report.get("colliding_particles", 0) + 1
        else:
            cost_o, g_o = orc.match_terms(p, th, st["nn_idx"][pk])
        assert abs(st["cost"][pk] - cost_o) <= COST_GRAD_REL * abs(cost_o) + COST_ABS, \
            f"particle {pk}: cost {st['cost'][pk]} vs {cost_o}"
        for blk in (slice(0, 3), slice(3, 7)):
            e = rel_err(st["grad"][pk, blk], g_o[blk], floor=1e-300)
            report["max_grad_rel"] = max(report.get("max_grad_rel", 0.0), e)
            assert np.linalg.norm(st["grad"][pk, blk] - g_o[blk]) <= COST_GRAD_REL * np.linalg.norm(g_o[blk]) + GRAD_ABS, \
                f"particle {pk}: gradient block {blk} relative error {e:.3e}"
        report["max_cost_rel"] = max(report.get("max_cost_rel", 0.0), abs(st["cost"][pk] - cost_o) / abs(cost_o))
    report["particles"] = report.get("particles", 0) + len(list(pks))
    if not check_update:
        return flips
    if sample is not None:
        # an SGD step moves each particle by its own gradient alone: check the sampled ones
        if k >= w.k_stein:
            for pk in pks:
                th = before_theta[pk].astype(np.float64)
                if st["frozen"][pk]:
                    assert np.array_equal(st["theta"][pk], before_theta[pk]), f"frozen particle {pk} moved"
                    continue
                new = th - st["grad"][pk]
                new[3:] /= np.linalg.norm(new[3:])
                err = np.abs(st["theta"][pk].astype(np.float64) - new).max()
                report["max_update_abs"] = max(report.get("max_update_abs", 0.0), err)
                assert err <= 2e-6, f"particle {pk}: updated pose differs by {err:.3e}"
        return flips
    # update: oracle's Stein / SGD step applied to the GPU's gradients (same pairs)
    svgd = k < w.k_stein
    for p in range(P):
        sl = slice(p * K, (p + 1) * K)
        th = before_theta[sl].astype(np.float64)
        if svgd:
            gam = oracle.gamma(k, w.k_max, w.schedule, w.C_cycles, w.p_exp, w.g0, w.g1)
            h = oracle.bandwidth(th)
            assert abs(st["h"][p] - h) <= 1e-5 * h, f"bandwidth {st['h'][p]} vs {h}"
            phi = oracle.stein_direction(th, st["grad"][sl], N, gam, h, prior=prior)
            scale = stein_term_scale(th, st["grad"][sl], N, gam, h, prior)
            for j in range(K):
                for b, blk in enumerate((slice(0, 3), slice(3, 7))):
                    e = np.linalg.norm(st["phi"][sl][j, blk] - phi[j, blk])
                    # relative error, with a floor for sums that cancel: float32 summation of K terms
                    # of magnitude `scale` carries an absolute error of ~sqrt(K) * 6e-8 * scale
                    tol = COST_GRAD_REL * np.linalg.norm(phi[j, blk]) + STEIN_ABS_REL * scale[j, b]
                    report["max_phi_err_over_tol"] = max(report.get("max_phi_err_over_tol", 0.0), e / tol)
                    assert e <= tol, f"preshape {p} particle {j}: Stein direction error {e:.3e} > {tol:.3e}"
            new = th + phi / N
        else:
            new = th - st["grad"][sl]
        new[:, 3:] /= np.linalg.norm(new[:, 3:], axis=1, keepdims=True)
        if not svgd:
            # converged particles keep their pose exactly (Table I criterion, Section IV-D)
            fr = np.asarray(st["frozen"][sl]).astype(bool)
            assert np.array_equal(st["theta"][sl][fr], before_theta[sl][fr]), "a frozen particle moved"
            new[fr] = before_theta[sl][fr]
        err = np.abs(st["theta"][sl].astype(np.float64) - new).max()
        report["max_update_abs"] = max(report.get("max_update_abs", 0.0), err)
        assert err <= 2e-6, f"preshape {p}: updated poses differ by {err:.3e}"
    return flips


STEIN_ABS_REL = 1e-5


def stein_term_scale(theta, grad, N, gam, h, prior=None):
    """Mean magnitude of the terms the Stein direction of each particle sums (per block)."""
    t, q = theta[:, :3], theta[:, 3:]
    dt = t[:, None, :] - t[None, :, :]                       # [i, j]
    kt = np.exp(-(dt ** 2).sum(-1) / h)
    c = np.abs(q @ q.T)
    pt = np.zeros(len(t)) if prior is None or prior[0] <= 0 else np.linalg.norm(t - prior[3], axis=1) / prior[0] ** 2
    pq = 0.0 if prior is None or prior[1] <= 0 else prior[1]
    st = (kt * (gam * N * np.linalg.norm(grad[None, :, :3], axis=-1) + gam * pt[None, :] +
                (2 / h) * np.linalg.norm(dt, axis=-1))).mean(1)
    sq = (c * (gam * N * np.linalg.norm(grad[None, :, 3:], axis=-1) + gam * pq) + 1.0).mean(1)
    return np.stack([st, sq], 1)


def geodesic_angle(q1, q2):
    """Rotation angle between unit quaternions (q and -q alike): 2 atan2(|q1 - s q2|, |q1 + s q2|) with
    s = sign(q1.q2), accurate down to the rounding of the inputs (arccos of the dot product is not:
    near 1 it magnifies float32 rounding to ~3e-4 rad)."""
    a = np.asarray(q1, np.float64)
    b = np.asarray(q2, np.float64)
    a = a / np.linalg.norm(a, axis=-1, keepdims=True)
    b = b / np.linalg.norm(b, axis=-1, keepdims=True)
    s = np.where((a * b).sum(-1) < 0, -1.0, 1.0)[..., None]
    return 2 * np.arctan2(np.linalg.norm(a - s * b, axis=-1), np.linalg.norm(a + s * b, axis=-1))


# Free-running runs: a particle whose trajectory came within FLIP_MARGIN (metres) of changing one
# of its discrete decisions (a correspondence, a collision flag, a reverse match: the oracle's
# decision margin) or within FREEZE_MARGIN (relative) of the convergence criterion may fork between
# the float32 GPU path and the FP64 oracle; those particles are reported separately, every other
# one must end within POSE_TOL_M / POSE_TOL_RAD of the oracle.
FLIP_MARGIN = 1e-6
FREEZE_MARGIN = 1e-3
POSE_TOL_M = 1e-3
POSE_TOL_RAD = 1e-3


def oracle_free_run(orc, theta0, sched, nthreads=1, conv_tol=-1.0):
    """Run the oracle free from theta0 (P, K, 7) for sched.k_max steps plus the final evaluation.
    Returns (state, trajectory, near_freeze): the poses at which every step (and the final
    evaluation) took its decisions, [k_max + 1] arrays (P, K, 7), and per particle whether a
    convergence decision came within FREEZE_MARGIN of the criterion."""
    st = orc.new_state(theta0)
    P, K = st["theta"].shape[:2]
    traj = []
    near_freeze = np.zeros((P, K), bool)
    for k in range(sched.k_max):
        prev = st["prev_cost"].copy()
        traj.append(st["theta"].copy())
        orc.step(st, sched, k, nthreads)
        if conv_tol >= 0 and k >= sched.k_stein:
            ok = (prev > 0) & (st["ncol"] == 0)
            rel = np.abs(st["cost"] - prev) / np.where(ok, prev, 1.0)
            near_freeze |= ok & (np.abs(rel - conv_tol) <= FREEZE_MARGIN * conv_tol)
    traj.append(st["theta"].copy())
    orc.evaluate(st, nthreads)
    return st, traj, near_freeze


def trajectory_margin(orc, traj, p, j):
    """Smallest decision margin (metres) of particle j of preshape p along an oracle trajectory."""
    return min(orc.decision_margin(p, th[p, j]) for th in traj)


def compare_final_poses(th_gpu, th_orc, orc, traj, near_freeze, label="", preshapes=None):
    """Final poses of a free run against the oracle's: a particle outside POSE_TOL_M / POSE_TOL_RAD
    passes only if its oracle trajectory took a decision within FLIP_MARGIN of a tie (or of the
    convergence criterion), and is reported as such.  preshapes: the oracle preshape index of each
    row (default: row // K).  Returns (position error, angle error, near-tie mask)."""
    th_gpu = np.asarray(th_gpu, np.float64).reshape(-1, 7)
    th_orc = np.asarray(th_orc, np.float64).reshape(-1, 7)
    P, K = traj[0].shape[:2]
    dpos = np.linalg.norm(th_gpu[:, :3] - th_orc[:, :3], axis=1)
    dang = geodesic_angle(th_gpu[:, 3:], th_orc[:, 3:])
    ok = (dpos <= POSE_TOL_M) & (dang <= POSE_TOL_RAD)
    tie = np.asarray(near_freeze).reshape(-1).copy()
    margins = {}
    for i in np.nonzero(~ok & ~tie)[0]:
        m = trajectory_margin(orc, traj, i // K, i % K)
        margins[int(i)] = m
        tie[i] = m < FLIP_MARGIN
    q = [0.5, 0.9, 0.99, 1.0]
    print(f"{label} final poses: {len(dpos)} particles, {int((~ok).sum())} outside tolerance, of which "
          f"{int((tie & ~ok).sum())} took a near-tie decision; position m (median, p90, p99, max) "
          f"{np.quantile(dpos, q)}, angle rad {np.quantile(dang, q)}")
    bad = np.nonzero(~ok & ~tie)[0]
    assert len(bad) == 0, (f"{label}: {len(bad)} particles without a near-tie decision differ beyond "
                           f"{POSE_TOL_M} m / {POSE_TOL_RAD} rad, e.g. {bad[:5]}: {dpos[bad[:5]]} m, "
                           f"{dang[bad[:5]]} rad, trajectory margins {[margins[int(i)] for i in bad[:5]]}")
    return dpos, dang, tie & ~ok
