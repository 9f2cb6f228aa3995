"""The proposal network's CUDA kernels (through include/asicp_proposal.h) against the FP64
oracle (oracle/proposal.py): forward outputs, loss, parameter gradients, the Adam step and
sampling.

Tolerances: both sides round the weights and the stored activations to bfloat16; the GPU
sums in float32 and the oracle exactly, so an activation can land on the other side of a
bfloat16 rounding boundary (one bfloat16 ulp, 2^-8 relative) and, rarely, a max-pool can pick
another point.  Outputs and gradients are therefore compared by norms: <= 2 % relative per
layer, cosine >= 0.999; the loss within 1e-3 relative."""
import numpy as np
import pytest

from paper_2412_08346_gb300 import proposal, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from oracle import proposal as orc  # noqa: E402

P, NPTS, T = 3, 256, 12


def _batch(B, seed):
    g = np.random.default_rng(seed)
    clouds = np.stack([synth.partial_object(NPTS, seed + 100 * b).points for b in range(B)]).astype(np.float32)
    tg = np.zeros((B, P, T, 7), np.float32)
    tg[..., :3] = clouds.mean(1)[:, None, None, :] + g.normal(0, 0.06, (B, P, T, 3))
    q = g.normal(size=(B, P, T, 4))
    tg[..., 3:] = q / np.linalg.norm(q, axis=-1, keepdims=True)
    return clouds, tg


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.fixture(scope="module")
def net():
    n = proposal.Proposal(P, NPTS, 8, torch.cuda.current_stream().cuda_stream)
    yield n
    n.close()


def test_forward_matches_oracle(net):
    params = synth.proposal_params(P, 11)
    params[orc.num_params(P) - P * 160:] = np.random.default_rng(3).normal(0, 0.5, P * 160)   # non-zero b5
    net.set_params(params)
    clouds, _ = _batch(4, 21)
    out, cen = net.forward(clouds, 4)
    for b in range(4):
        o, _, c = orc.forward(params, clouds[b], P)
        assert np.allclose(cen[b], c, rtol=0, atol=1e-6)
        assert _rel(out[b], o) <= 0.02, f"object {b}: {_rel(out[b], o):.3e}"


def test_loss_and_gradient_match_oracle(net):
    params = synth.proposal_params(P, 12)
    net.set_params(params)
    clouds, tg = _batch(4, 31)
    loss, grad = net.loss_grad(clouds, tg, 4, T, want_grad=True)
    lo, go = orc.loss_and_grad(params, list(clouds), list(tg), P)
    assert abs(loss - lo) <= 1e-3 * abs(lo), (loss, lo)
    start = 0
    for (o, i) in orc.layer_shapes(P):
        for n in (o * i, o):
            a, b = grad[start:start + n], go[start:start + n]
            cos = float(a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30))
            assert _rel(a, b) <= 0.02 and cos >= 0.999, (start, n, _rel(a, b), cos)
            start += n


def test_adam_step_matches_oracle(net):
    params = synth.proposal_params(P, 13)
    net.set_params(params)
    clouds, tg = _batch(2, 41)
    _, grad = net.loss_grad(clouds, tg, 2, T, want_grad=True)
    net.adam_step(1e-3)
    got = net.get_params()
    ref, _, _ = orc.adam(params.astype(np.float64), grad.astype(np.float64), np.zeros_like(grad, np.float64),
                         np.zeros_like(grad, np.float64), 1, 1e-3)
    assert np.allclose(got, ref, rtol=0, atol=1e-6)


def test_sampling_matches_oracle(net):
    params = synth.proposal_params(P, 14)
    params[orc.num_params(P) - P * 160:] = np.random.default_rng(5).normal(0, 1.0, P * 160)
    net.set_params(params)
    clouds, _ = _batch(2, 51)
    out, cen = net.forward(clouds, 2)
    K = 64
    g = np.random.default_rng(6)
    draws = np.concatenate([g.uniform(0, 1, (2, P, K, 1)), g.normal(size=(2, P, K, 7))], -1).astype(np.float32)
    th = net.sample(out, cen, 2, K, draws)
    flips = 0
    for b in range(2):
        for p in range(P):
            ref = orc.sample(out[b, p].astype(np.float64), cen[b].astype(np.float64), draws[b, p].astype(np.float64))
            err = np.abs(th[b, p] - ref).max(1)
            flips += int((err > 1e-4).sum())       # a draw on a component boundary may pick the neighbour
    assert flips <= 2
    assert np.allclose(np.linalg.norm(th[..., 3:], axis=-1), 1.0, atol=1e-5)


def test_training_reduces_the_loss(net):
    net.set_params(synth.proposal_params(P, 15))
    clouds, tg = _batch(8, 61)
    first, _ = net.loss_grad(clouds, tg, 8, T)
    for _ in range(60):
        net.loss_grad(clouds, tg, 8, T)
        net.adam_step(3e-3)
    last, _ = net.loss_grad(clouds, tg, 8, T)
    assert last < first - 0.5, (first, last)


def test_trained_proposal_generalises_to_held_out_objects():
    """Targets from the plain method on procedural objects; after training, the loss on held-out
    objects is well below the untrained network's (the network has learned where good grasps of
    unseen objects lie), and its samples feed asicp_run."""
    from paper_2412_08346_gb300 import asicp, learned_init
    stream = torch.cuda.current_stream().cuda_stream
    npts = 1024
    pre = synth.make_preshapes(3, 512, 32, synth.BASE_SEED + 9)
    train_c = learned_init.object_clouds(160, npts, synth.BASE_SEED + 70_000)
    test_c = learned_init.object_clouds(32, npts, synth.BASE_SEED + 80_000)
    tg_train, _ = learned_init.converged_targets(train_c, pre, K=96, k_max=40, stream=stream)
    tg_test, _ = learned_init.converged_targets(test_c, pre, K=96, k_max=40, stream=stream)
    net = proposal.Proposal(3, npts, 32, stream)
    try:
        net.set_params(synth.proposal_params(3, 17))
        before, _ = net.loss_grad(test_c, tg_test, 32, tg_test.shape[2])
        hist = learned_init.train(net, train_c, tg_train, epochs=40, batch=32, lr=1e-3, seed=3)
        after, _ = net.loss_grad(test_c, tg_test, 32, tg_test.shape[2])
        print(f"held-out loss {before:.3f} -> {after:.3f}; training {hist[0]:.3f} -> {hist[-1]:.3f}")
        assert after < before - 1.0
        th0, _ = learned_init.propose(net, test_c[:4], 32, seed=1)
        best, _ = learned_init.run_grasp_sets(test_c[:4], pre, 32, 10, stream, theta0=th0, batch=4)
        assert np.all(np.isfinite(best))
    finally:
        net.close()
