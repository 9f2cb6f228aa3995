"""FP64 oracle of the learned initial-pose proposal (test infrastructure only).

The paper initialises particles on a Fibonacci sphere, shows that initialising
from a mixture of Gaussians placed with prior knowledge of the object needs fewer
particles for the same success rate (Section VII ablation, Fig. 3 and its
discussion), and names learned initial poses as future work (Conclusions).  The
proposal network below fills that slot: a PointNet-style encoder maps the
object cloud to a mixture of SE(3) densities per preshape, trained on the
converged particle sets of the plain method.  This module writes every step
out in float64 numpy so that the CUDA kernels can be checked against it.

Network (weights row-major [out][in]; x_i = r_i - centroid):
    h1_i = relu(W1 x_i + b1)          3 -> 64
    h2_i = relu(W2 h1_i + b2)        64 -> 128
    h3_i = relu(W3 h2_i + b3)       128 -> 256
    g    = max_i h3_i (per channel; ties to the lowest point index)
    z    = relu(W4 g + b4)          256 -> 256
    o    = W5 z + b5                256 -> P * C * 9
Weights, the centred input and the stored activations (h1, h2, h3, g, z) are
bfloat16 values (round to nearest even); products and sums are exact here and
float32 on the GPU.

Mixture (per preshape p, component c; raw outputs o[p, c, 0..9]):
    pi_c    = softmax_c(o0)
    mu_c    = 0.1 (o1, o2, o3)                     translation relative to the centroid
    sigma_c = 0.1 exp(clip(o4, -4, 1))             isotropic translation spread
    nu_c    = (o5..o8) / max(|o5..o8|, 1e-6)       rotation mean (unit quaternion)
    kappa_c = 4 exp(clip(o9, -2, 3))               rotational concentration
    log p(t, q) = LSE_c [log pi_c - |t' - mu_c|^2 / (2 sigma_c^2) - 3 log sigma_c
                         + kappa_c (nu_c . q)^2 - log M(1/2, 2, kappa_c)]
                  - 1.5 log(2 pi) - log(2 pi^2)
with t' = t - centroid: a Gaussian in translation times a Watson density on the
quaternion sphere S^3 (so q and -q score alike), M = Kummer's confluent
hypergeometric function 1F1 (the Watson normaliser; d/dk log M(1/2, 2, k) =
M(3/2, 3, k) / (4 M(1/2, 2, k))) and 2 pi^2 the area of S^3.
Loss of one object: L = -(1 / (P T)) sum_p sum_j log p_p(t_pj, q_pj) over T
target poses per preshape.
"""
from __future__ import annotations

import numpy as np

C_COMP = 16          # mixture components per preshape
N_RAW = 10           # raw outputs per component
HIDDEN = (64, 128, 256)
HEAD = 256


def layer_shapes(P: int):
    """(out, in) of W1..W5; biases have length out."""
    return [(HIDDEN[0], 3), (HIDDEN[1], HIDDEN[0]), (HIDDEN[2], HIDDEN[1]), (HEAD, HIDDEN[2]),
            (P * C_COMP * N_RAW, HEAD)]


def num_params(P: int) -> int:
    return sum(o * i + o for o, i in layer_shapes(P))


def unflatten(flat: np.ndarray, P: int):
    """Flat layout: W1, b1, W2, b2, ..., W5, b5 (W row-major [out][in])."""
    out, k = [], 0
    for o, i in layer_shapes(P):
        W = flat[k:k + o * i].reshape(o, i); k += o * i
        b = flat[k:k + o]; k += o
        out.append((W, b))
    assert k == flat.size
    return out


def flatten(layers) -> np.ndarray:
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in layers])


def bf16(x: np.ndarray) -> np.ndarray:
    """Round float64 values to the nearest bfloat16 (8-bit significand, float32's exponent range,
    ties to even), returned as float64: one rounding from the float64 value, with the spacing
    2^(e-8) of the binade [2^(e-1), 2^e) (2^-133 below the normal range)."""
    x = np.asarray(x, dtype=np.float64)
    _, e = np.frexp(x)
    e = np.maximum(e, -125)
    return np.ldexp(np.rint(np.ldexp(x, 8 - e)), e - 8)


def forward(flat: np.ndarray, cloud: np.ndarray, P: int, round_bf16: bool = True):
    """One object: returns (o [P, C, 9], cache for backward, centroid).  round_bf16=False
    keeps every value in float64 (for finite-difference checks of the backward pass)."""
    rb = bf16 if round_bf16 else (lambda a: np.asarray(a, np.float64))
    layers = unflatten(np.asarray(flat, np.float64), P)
    Wq = [(rb(W), np.asarray(b, np.float64)) for W, b in layers]   # weights bf16, biases float32
    r = np.asarray(cloud, np.float64)
    cen = r.mean(0)
    x = rb(np.asarray(r - cen, np.float32) if round_bf16 else r - cen)
    h1 = rb(np.maximum(x @ Wq[0][0].T + Wq[0][1], 0.0))
    h2 = rb(np.maximum(h1 @ Wq[1][0].T + Wq[1][1], 0.0))
    h3 = rb(np.maximum(h2 @ Wq[2][0].T + Wq[2][1], 0.0))
    arg = np.argmax(h3, axis=0)                     # first maximum = lowest point index
    gmax = h3[arg, np.arange(h3.shape[1])]
    z = rb(np.maximum(gmax @ Wq[3][0].T + Wq[3][1], 0.0))
    o = z @ Wq[4][0].T + Wq[4][1]
    cache = dict(x=x, h1=h1, h2=h2, h3=h3, arg=arg, g=gmax, z=z, W=Wq)
    return o.reshape(P, C_COMP, N_RAW), cache, cen


def log_kummer(k):
    """log M(1/2, 2, k) and its derivative (scipy's 1F1)."""
    from scipy.special import hyp1f1
    m = hyp1f1(0.5, 2.0, k)
    return np.log(m), 0.25 * hyp1f1(1.5, 3.0, k) / m


def mixture(o: np.ndarray):
    """Mixture parameters of one preshape from its raw outputs o [C, 10]."""
    a = o[:, 0]
    logpi = a - (a.max() + np.log(np.exp(a - a.max()).sum()))
    mu = 0.1 * o[:, 1:4]
    s = np.clip(o[:, 4], -4.0, 1.0)
    sigma = 0.1 * np.exp(s)
    v = o[:, 5:9]
    nv = np.maximum(np.linalg.norm(v, axis=1), 1e-6)
    nu = v / nv[:, None]
    kappa = 4.0 * np.exp(np.clip(o[:, 9], -2.0, 3.0))
    return logpi, mu, sigma, nu, kappa


CONST = -1.5 * np.log(2 * np.pi) - np.log(2 * np.pi ** 2)


def log_density(o: np.ndarray, t_rel: np.ndarray, q: np.ndarray) -> np.ndarray:
    """log p(t, q) of one preshape's mixture at poses (t relative to the centroid)."""
    logpi, mu, sigma, nu, kappa = mixture(o)
    lm, _ = log_kummer(kappa)
    d2 = ((t_rel[:, None, :] - mu[None, :, :]) ** 2).sum(-1)
    dot = q @ nu.T
    ell = logpi[None, :] - d2 / (2 * sigma[None, :] ** 2) - 3 * np.log(sigma)[None, :] + kappa * dot ** 2 - lm
    m = ell.max(1, keepdims=True)
    return (m + np.log(np.exp(ell - m).sum(1, keepdims=True)))[:, 0] + CONST


def loss_and_grad_o(o: np.ndarray, targets: np.ndarray, cen: np.ndarray):
    """Loss of one object and its gradient with respect to the raw outputs.

    o [P, C, 9]; targets [P, T, 7] (t, q) in the object frame."""
    P, T = targets.shape[0], targets.shape[1]
    loss = 0.0
    go = np.zeros_like(o)
    for p in range(P):
        t = targets[p, :, :3] - cen
        q = targets[p, :, 3:7]
        logpi, mu, sigma, nu, kappa = mixture(o[p])
        lm, dlm = log_kummer(kappa)
        diff = t[:, None, :] - mu[None, :, :]                          # [T, C, 3]
        d2 = (diff ** 2).sum(-1)
        dot = q @ nu.T
        ell = logpi[None, :] - d2 / (2 * sigma ** 2) - 3 * np.log(sigma) + kappa * dot ** 2 - lm
        m = ell.max(1, keepdims=True)
        lse = m[:, 0] + np.log(np.exp(ell - m).sum(1))
        loss -= (lse + CONST).sum()
        r = np.exp(ell - lse[:, None])                                  # responsibilities [T, C]
        pi = np.exp(logpi)
        w = -1.0 / (P * T)
        # d(-log p)/d ell_c = -r_c; ell_c depends on the logits through log pi
        go[p, :, 0] += w * (r.sum(0) - T * pi)
        dmu = (r[:, :, None] * diff / (sigma[None, :, None] ** 2)).sum(0)          # d ell / d mu
        go[p, :, 1:4] += w * 0.1 * dmu
        dsig = (r * (d2 / sigma ** 3 - 3.0 / sigma)).sum(0)
        inside = (o[p, :, 4] > -4.0) & (o[p, :, 4] < 1.0)
        go[p, :, 4] += w * np.where(inside, dsig * sigma, 0.0)
        dnu = (r[:, :, None] * (2 * kappa[None, :, None] * dot[:, :, None]) * q[:, None, :]).sum(0)   # [C, 4]
        v = o[p, :, 5:9]
        nv = np.maximum(np.linalg.norm(v, axis=1), 1e-6)
        proj = dnu - (dnu * nu).sum(1, keepdims=True) * nu
        go[p, :, 5:9] += w * proj / nv[:, None]
        dkap = (r * (dot ** 2 - dlm[None, :])).sum(0)
        kin = (o[p, :, 9] > -2.0) & (o[p, :, 9] < 3.0)
        go[p, :, 9] += w * np.where(kin, dkap * kappa, 0.0)
    return loss / (P * T), go


def backward(go: np.ndarray, cache: dict, P: int) -> np.ndarray:
    """Gradient of the loss with respect to the flat parameters (through the bf16 weights,
    whose rounding is treated as the identity for the gradient, as on the GPU)."""
    (W1, _), (W2, _), (W3, _), (W4, _), (W5, _) = cache["W"]
    x, h1, h2, h3, arg, g, z = (cache[k] for k in ("x", "h1", "h2", "h3", "arg", "g", "z"))
    do = go.reshape(-1)
    dW5 = np.outer(do, z); db5 = do
    dz = (W5.T @ do) * (z > 0)
    dW4 = np.outer(dz, g); db4 = dz
    dg = W4.T @ dz
    dh3 = np.zeros_like(h3)
    dh3[arg, np.arange(h3.shape[1])] = dg
    dh3 = dh3 * (h3 > 0)
    dW3 = dh3.T @ h2; db3 = dh3.sum(0)
    dh2 = (dh3 @ W3) * (h2 > 0)
    dW2 = dh2.T @ h1; db2 = dh2.sum(0)
    dh1 = (dh2 @ W2) * (h1 > 0)
    dW1 = dh1.T @ x; db1 = dh1.sum(0)
    return flatten([(dW1, db1), (dW2, db2), (dW3, db3), (dW4, db4), (dW5, db5)])


def loss_and_grad(flat: np.ndarray, clouds, targets, P: int, round_bf16: bool = True):
    """Mean loss over a batch of objects and its gradient (flat)."""
    total, grad = 0.0, np.zeros(num_params(P))
    for cloud, tg in zip(clouds, targets):
        o, cache, cen = forward(flat, cloud, P, round_bf16)
        l, go = loss_and_grad_o(o, tg, cen)
        total += l
        grad += backward(go, cache, P)
    n = len(clouds)
    return total / n, grad / n


def adam(flat, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (float64); returns new (flat, m, v)."""
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** step)
    vh = v / (1 - b2 ** step)
    return flat - lr * mh / (np.sqrt(vh) + eps), m, v


def sample(o: np.ndarray, cen: np.ndarray, draws: np.ndarray) -> np.ndarray:
    """Initial poses from one preshape's mixture: draws [K, 8] = (u, n1..n7) with u uniform in
    [0, 1) picking the component by its cumulative weight, n standard normal.
    t = centroid + mu_c + sigma_c (n1, n2, n3); q = normalise(nu_c + (n4..n7) / sqrt(2 kappa_c))
    (a Gaussian perturbation of the mean axis: close to the Watson density for large kappa)."""
    logpi, mu, sigma, nu, kappa = mixture(o)
    cdf = np.cumsum(np.exp(logpi))
    out = np.zeros((draws.shape[0], 7))
    for k, d in enumerate(draws):
        c = int(np.searchsorted(cdf, d[0] * cdf[-1], side="right"))
        c = min(c, C_COMP - 1)
        t = cen + mu[c] + sigma[c] * d[1:4]
        q = nu[c] + d[4:8] / np.sqrt(2 * kappa[c])
        out[k, :3] = t
        out[k, 3:] = q / np.linalg.norm(q)
    return out
