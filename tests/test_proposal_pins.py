"""Pins of the proposal-network oracle (oracle/proposal.py) against closed forms,
finite differences and library routines."""
import numpy as np
import pytest

from oracle import proposal as pr
from paper_2412_08346_gb300 import synth


def _rand_targets(g, P, T):
    t = g.normal(0, 0.08, (P, T, 3))
    q = g.normal(size=(P, T, 4))
    q /= np.linalg.norm(q, axis=2, keepdims=True)
    return np.concatenate([t, q], 2)


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1 + 2 ** -9, 1 + 3 * 2 ** -9, -2.5, 3.0e-3, 0.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8])
    got = pr.bf16(vals)
    # 8-bit significand: ulp(1) = 2^-7; 1 + 2^-8 and 1 + 3 * 2^-8 are ties -> the even neighbour
    assert got[0] == 1.0 and got[1] == 1.0 and got[2] == 1 + 2 ** -7 and got[3] == -2.5 and got[5] == 0.0
    assert got[6] == 1.0 and got[7] == 1 + 2 ** -6
    assert abs(got[4] - 3.0e-3) <= 2 ** -8 * 3.0e-3
    # one rounding from float64: a value just above a tie goes up although its float32 rounding
    # lands exactly on the tie (which would then go to the even neighbour)
    just_above = 1 + 2 ** -8 + 2 ** -40
    assert np.float32(just_above) == np.float32(1 + 2 ** -8)
    assert pr.bf16(np.array([just_above]))[0] == 1 + 2 ** -7
    # against a bit-level reference on random float32 values (exact in float64): same result
    g = np.random.default_rng(1)
    f = (g.normal(size=2000) * np.exp(g.uniform(-30, 30, 2000))).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    ref = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)
    assert np.array_equal(pr.bf16(f.astype(np.float64)), ref.astype(np.float64))
    # below float32's normal range the spacing is 2^-133
    assert pr.bf16(np.array([3 * 2.0 ** -134]))[0] == 2 * 2.0 ** -133


def test_single_component_density_is_gaussian_times_watson():
    """With one logit dominating, p = N(t; mu, sigma^2 I) x Watson(q; nu, kappa) on S^3."""
    from scipy.special import hyp1f1
    from scipy.stats import multivariate_normal
    g = np.random.default_rng(1)
    o = g.normal(size=(pr.C_COMP, pr.N_RAW))
    o[:, 0] = -80.0
    o[3, 0] = 80.0
    logpi, mu, sigma, nu, kappa = pr.mixture(o)
    t = g.normal(0, 0.05, (5, 3))
    q = g.normal(size=(5, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    watson = np.exp(kappa[3] * (q @ nu[3]) ** 2) / (hyp1f1(0.5, 2.0, kappa[3]) * 2 * np.pi ** 2)
    ref = multivariate_normal(mu[3], sigma[3] ** 2 * np.eye(3)).logpdf(t) + np.log(watson)
    assert np.allclose(pr.log_density(o, t, q), ref, rtol=0, atol=1e-9)


def test_rotation_factor_integrates_to_one_on_s3():
    """Monte Carlo over uniform unit quaternions: E[exp(kappa (nu.q)^2) / M(1/2, 2, kappa)] = 1."""
    g = np.random.default_rng(11)
    q = g.normal(size=(400000, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    nu = np.array([0.5, -0.5, 0.5, 0.5])
    for kappa in (0.6, 4.0, 15.0):
        lm, dlm = pr.log_kummer(np.array([kappa]))
        mean = np.exp(kappa * (q @ nu) ** 2 - lm[0]).mean()
        assert abs(mean - 1.0) < 0.02 * max(1.0, np.sqrt(kappa)), (kappa, mean)
        h = 1e-5    # the derivative of log M against central differences
        fd = (pr.log_kummer(np.array([kappa + h]))[0][0] - pr.log_kummer(np.array([kappa - h]))[0][0]) / (2 * h)
        assert abs(fd - dlm[0]) < 1e-7


def test_density_is_antipodal_invariant():
    g = np.random.default_rng(2)
    o = g.normal(size=(pr.C_COMP, pr.N_RAW))
    t = g.normal(0, 0.05, (7, 3))
    q = g.normal(size=(7, 4)); q /= np.linalg.norm(q, axis=1, keepdims=True)
    assert np.allclose(pr.log_density(o, t, q), pr.log_density(o, t, -q), rtol=0, atol=1e-12)


def test_output_gradient_matches_finite_differences():
    g = np.random.default_rng(3)
    P, T = 2, 5
    o = g.normal(size=(P, pr.C_COMP, pr.N_RAW))
    o[..., 4] = g.uniform(-3.5, 0.5, (P, pr.C_COMP))          # inside the clip ranges
    o[..., 9] = g.uniform(-1.5, 2.5, (P, pr.C_COMP))
    tg = _rand_targets(g, P, T)
    cen = g.normal(0, 0.01, 3)
    _, go = pr.loss_and_grad_o(o, tg, cen)
    h = 1e-6
    for idx in [(0, 0, 0), (1, 5, 2), (0, 7, 4), (1, 3, 6), (0, 15, 8), (1, 9, 1), (0, 4, 9), (1, 12, 9)]:
        op, om = o.copy(), o.copy()
        op[idx] += h; om[idx] -= h
        fd = (pr.loss_and_grad_o(op, tg, cen)[0] - pr.loss_and_grad_o(om, tg, cen)[0]) / (2 * h)
        assert abs(fd - go[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, go[idx])


def test_parameter_gradient_matches_finite_differences():
    """Backward pass of the whole network (float64, no bf16 rounding) against central differences."""
    g = np.random.default_rng(4)
    P = 1
    flat = synth.proposal_params(P, 5).astype(np.float64)
    clouds = [g.normal(0, 0.05, (40, 3)) + 0.2, g.normal(0, 0.04, (40, 3))]
    tgs = [_rand_targets(g, P, 4), _rand_targets(g, P, 4)]
    _, grad = pr.loss_and_grad(flat, clouds, tgs, P, round_bf16=False)
    sizes = [o * i + o for o, i in pr.layer_shapes(P)]
    starts = np.cumsum([0] + sizes)
    h = 1e-6
    picks = [starts[L] + k for L in range(5) for k in (0, sizes[L] // 2, sizes[L] - 1)]
    for j in picks:
        fp, fm = flat.copy(), flat.copy()
        fp[j] += h; fm[j] -= h
        fd = (pr.loss_and_grad(fp, clouds, tgs, P, round_bf16=False)[0] -
              pr.loss_and_grad(fm, clouds, tgs, P, round_bf16=False)[0]) / (2 * h)
        assert abs(fd - grad[j]) <= 1e-5 * max(1e-3, abs(fd)) + 1e-9, (j, fd, grad[j])


def test_maxpool_ties_go_to_the_lowest_point():
    P = 1
    flat = synth.proposal_params(P, 6).astype(np.float64)
    cloud = np.zeros((8, 3))          # every point identical: every channel ties across points
    cloud[:, 0] = 0.1
    _, cache, _ = pr.forward(flat, cloud, P)
    assert np.all(cache["arg"] == 0)


def test_adam_first_step_is_a_signed_unit_step():
    g = np.random.default_rng(7)
    w = g.normal(size=20)
    grad = g.normal(size=20)
    nw, m, v = pr.adam(w, grad, np.zeros(20), np.zeros(20), 1, 0.01, eps=0.0)
    assert np.allclose(nw, w - 0.01 * np.sign(grad), rtol=0, atol=1e-15)


def test_sampling_follows_the_mixture():
    """Component frequencies ~ pi, translation mean of a component ~ centroid + mu."""
    g = np.random.default_rng(8)
    o = g.normal(size=(pr.C_COMP, pr.N_RAW))
    o[:, 0] = -50.0
    o[2, 0] = 0.0
    o[9, 0] = np.log(3.0)             # two live components, weights 1/4 and 3/4
    o[2, 1:4] = (5.0, 0.0, 0.0)       # means 0.5 m apart along x, spread 5 mm
    o[9, 1:4] = (-5.0, 0.0, 0.0)
    o[[2, 9], 4] = -3.0
    cen = np.array([0.1, -0.2, 0.3])
    K = 20000
    draws = np.concatenate([g.uniform(0, 1, (K, 1)), g.normal(size=(K, 7))], 1)
    th = pr.sample(o, cen, draws)
    lab = th[:, 0] < cen[0]
    assert abs(lab.mean() - 0.75) < 0.02
    assert abs(th[lab, 0].mean() - (cen[0] - 0.5)) < 1e-3 and abs(th[~lab, 0].mean() - (cen[0] + 0.5)) < 1e-3
    assert np.allclose(np.linalg.norm(th[:, 3:], axis=1), 1.0)
