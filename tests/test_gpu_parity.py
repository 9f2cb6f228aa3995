"""CUDA path (through the C-ABI) against the FP64 oracle.

Teacher-forced single steps compare every output of the step on the same poses;
free-running runs compare final poses; the full-size workload is checked on
sampled particles; edge cases cover ragged tiles, tiny and degenerate sizes.
"""
import numpy as np
import pytest

from paper_2412_08346_gb300 import asicp, synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import asicp_testlib as tl  # noqa: E402


@pytest.fixture(scope="module")
def stream():
    return torch.cuda.current_stream().cuda_stream


def _ctx(w, stream, **over):
    cfg = tl.make_config(w, stream=stream, **over)
    return asicp.asicp_create(cfg)


def _teacher_forced_run(w, stream, steps, report, device=True, theta0=None, sample=None, **over):
    """Run `steps` GPU steps; before each, read the GPU's poses and compare the step with the oracle."""
    orc = tl.make_oracle(w)
    ctx = _ctx(w, stream, **over)
    try:
        keep = tl.upload(ctx, w, device=device)
        P, K, N, Mc = len(w.preshapes), w.K, w.preshapes[0].S.shape[0], len(w.objects[0].points)
        if theta0 is None:
            com = orc.R.mean(0)
            import oracle
            theta0 = np.tile(oracle.fibonacci_init(K, com, 0.15), (P, 1)).astype(np.float32)
        asicp.asicp_set_state(ctx, np.ascontiguousarray(theta0, dtype=np.float32), 0)
        for k in steps:
            asicp.asicp_set_state(ctx, tl.read_theta(ctx, P * K), k)
            before = tl.read_theta(ctx, P * K)      # the poses exactly as stored (set_state renormalises q)
            asicp.asicp_step(ctx, k)
            st = tl.read_state(ctx, P, K, N, Mc)
            tl.check_step(orc, w, before, st, k, report, sample=sample)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    return report


def test_small_box_teacher_forced_steps(stream):
    """1 preshape, K=32, N=256, M=512: every step of a 50-step trajectory, teacher-forced."""
    w = synth.small_box_case()
    rep = _teacher_forced_run(w, stream, range(w.k_max), {})
    print("small box:", rep)
    assert rep["nn_total"] == 50 * 32 * 256
    assert rep.get("nn_near_ties", 0) <= 1e-4 * rep["nn_total"]


def test_multi_preshape_ragged_tiles_with_collisions(stream):
    """3 preshapes, N=1000 (ragged query block), M=5000 (two full tiles + a ragged one), poses close to
    the object so collisions occur; SVGD and SGD phases."""
    w = synth.custom_case(P=3, K=24, N=1000, M=5000, grid=40, k_max=12, seed=7, k_stein=6)
    import oracle
    com = w.objects[0].points.astype(np.float64).mean(0)
    th = oracle.fibonacci_init(w.K, com, 0.05)          # 5 cm: fingers reach into the object
    theta0 = np.tile(th, (3, 1)).astype(np.float32)
    rep = _teacher_forced_run(w, stream, [0, 1, 2, 5, 6, 7, 11], {}, theta0=theta0)
    print("ragged + collisions:", rep)
    assert rep.get("colliding_particles", 0) > 0, "the case is meant to exercise the collision path"


def test_host_pointer_inputs_match_device_pointer_inputs(stream):
    w = synth.custom_case(P=2, K=16, N=300, M=700, grid=24, k_max=4, seed=11)
    outs = []
    for device in (True, False):
        ctx = _ctx(w, stream)
        try:
            keep = tl.upload(ctx, w, device=device)
            asicp.asicp_run(ctx)
            th = np.zeros((7 * 8,), np.float32)
            cost = np.zeros(8, np.float32)
            pre = np.zeros(8, np.int32)
            n = asicp.asicp_best_grasps(ctx, 8, th, cost, pre)
            assert n == 8
            outs.append((th.copy(), cost.copy(), pre.copy()))
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("shape", [0, asicp.FWD_SHAPES - 1])
def test_free_running_small_box_final_poses(stream, shape):
    """50 free-running iterations on both sides (float32 and tensor-core matching): every particle
    whose trajectory kept its discrete decisions clear of ties (decision margin >= 1 um all along)
    ends within 1 mm / 1e-3 rad of the oracle; near-tie particles are reported separately."""
    import oracle
    w = synth.small_box_case()
    orc = tl.make_oracle(w)
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, g0=w.g0, g1=w.g1, N=orc.N)
    theta0 = oracle.fibonacci_init(w.K, orc.R.mean(0), 0.15)
    ost, traj, near = tl.oracle_free_run(orc, theta0.astype(np.float32).astype(np.float64)[None], sched,
                                         nthreads=4)
    ctx = _ctx(w, stream, debug=False, fwd_shape=shape)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx, np.ascontiguousarray(theta0.astype(np.float32)))
        th = tl.read_theta(ctx, w.K)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    dpos, dang, tie = tl.compare_final_poses(th, ost["theta"][0], orc, traj, near, f"small box, shape {shape}")
    assert np.median(dpos) <= 1e-6


def test_paper_scale_sampled_step(stream):
    """3 x 256 particles, N=2048, M=8192, SDF 64^3: sampled particles of an SVGD and an SGD step from
    the initial poses, in the launch configuration the benchmark uses (the tensor-core matching
    shape, which the autotuner picks at this workload; the float32 shape is covered at this size as
    well), and a step from converged, partly colliding poses: the poses after 60 free-running
    iterations, teacher-forced one SGD step (colliding and free particles sampled)."""
    import oracle
    w = synth.paper_scale_case()
    g = np.random.default_rng(3)
    sample = sorted(g.choice(w.K * 3, 24, replace=False).tolist())
    rep = _teacher_forced_run(w, stream, [0, 60], {}, sample=sample, fwd_shape=asicp.FWD_SHAPES - 1)
    print("paper scale sampled (tensor cores):", rep)
    rep = _teacher_forced_run(w, stream, [0], {}, sample=sample[:8], fwd_shape=0)
    print("paper scale sampled:", rep)
    # converged poses: 60 free iterations on the GPU, then one teacher-forced step
    P, K, N, M = 3, w.K, 2048, 8192
    orc = tl.make_oracle(w)
    theta0 = np.tile(oracle.fibonacci_init(K, orc.R.mean(0), 0.15), (P, 1)).astype(np.float32)
    ctx = _ctx(w, stream, fwd_shape=asicp.FWD_SHAPES - 1)
    rep = {}
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_set_state(ctx, theta0, 0)
        for k in range(60):
            asicp.asicp_step(ctx, k)
        st = tl.read_state(ctx, P, K, N, M, debug=False)
        col = np.nonzero(st["ncol"] > 0)[0]
        free = np.nonzero(st["ncol"] == 0)[0]
        sample = sorted(set(g.choice(col, min(12, len(col)), replace=False).tolist()) |
                        set(g.choice(free, min(12, len(free)), replace=False).tolist()))
        asicp.asicp_set_state(ctx, tl.read_theta(ctx, P * K), 60)
        before = tl.read_theta(ctx, P * K)
        asicp.asicp_step(ctx, 60)
        st = tl.read_state(ctx, P, K, N, M)
        tl.check_step(orc, w, before, st, 60, rep, sample=sample)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    print("paper scale, converged poses (tensor cores):", rep, "colliding after 60 iterations:", len(col))
    assert rep.get("colliding_particles", 0) > 0, "the converged poses are meant to include collisions"


def test_single_particle_stein_equals_sgd(stream):
    """K = 1, gamma = 1: one SVGD step equals one SGD step (Eq. 8 reduces to Eq. 3)."""
    w = synth.custom_case(P=1, K=1, N=128, M=256, grid=16, k_max=2, seed=5)
    import oracle
    th0 = oracle.fibonacci_init(1, w.objects[0].points.astype(np.float64).mean(0), 0.08).astype(np.float32)
    res = []
    for k_stein in (2, 0):
        ctx = _ctx(w, stream, k_stein=k_stein, schedule=1, g0=1.0, g1=1.0)
        try:
            keep = tl.upload(ctx, w)
            asicp.asicp_set_state(ctx, th0, 0)
            asicp.asicp_step(ctx, 0)
            res.append(tl.read_theta(ctx, 1))
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    assert np.abs(res[0] - res[1]).max() <= 1e-6


def test_degenerate_sizes(stream):
    """M = 1 (every point pairs with the one object point), N = 1, K = 2."""
    w = synth.custom_case(P=1, K=2, N=1, M=1, grid=8, k_max=2, seed=13)
    rep = _teacher_forced_run(w, stream, [0, 1], {})
    assert rep["nn_total"] == 4


def test_selection_and_determinism(stream):
    w = synth.custom_case(P=2, K=32, N=256, M=1024, grid=24, k_max=8, seed=17)
    runs = []
    for _ in range(2):
        ctx = _ctx(w, stream)
        try:
            keep = tl.upload(ctx, w)
            asicp.asicp_run(ctx)
            st = tl.read_state(ctx, 2, 32, 256, 1024, debug=False)
            best = np.zeros(64 * 7, np.float32)
            cost = np.zeros(64, np.float32)
            pre = np.zeros(64, np.int32)
            asicp.asicp_best_grasps(ctx, 64, best, cost, pre)
            runs.append((st, best, cost, pre))
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    (a, ba, ca, pa), (b, bb, cb, pb) = runs
    for key in ("theta", "cost", "grad", "ncol"):
        assert np.array_equal(a[key], b[key]), f"{key} differs between identical runs"
    assert np.array_equal(ba, bb)
    import oracle
    order = oracle.select(a["cost"], a["ncol"], 64)
    assert np.array_equal(pa, order // 32)
    assert np.allclose(ca, a["cost"][order].astype(np.float32))
    assert np.array_equal(ba.reshape(64, 7), a["theta"][order])


def test_invalid_inputs_are_rejected(stream):
    w = synth.custom_case(P=1, K=4, N=16, M=32, grid=8, k_max=2, seed=19)
    ctx = _ctx(w, stream)
    try:
        with pytest.raises(asicp.AsicpError) as e:
            asicp.asicp_step(ctx, 0)
        assert e.value.status == asicp.ASICP_ERR_STATE
        bad = w.objects[0].points.copy()
        bad[3, 1] = np.nan
        with pytest.raises(asicp.AsicpError) as e:
            asicp.asicp_set_object(ctx, bad)
        assert e.value.status == asicp.ASICP_ERR_INVALID_ARG
        keep = tl.upload(ctx, w)
        with pytest.raises(asicp.AsicpError) as e:
            asicp.asicp_step(ctx, 0)            # poses not set yet
        assert e.value.status == asicp.ASICP_ERR_STATE
        with pytest.raises(asicp.AsicpError) as e:
            asicp.asicp_set_gripper_sdf(ctx, 0, w.preshapes[0].S, np.zeros((1, 8, 8), np.float32),
                                        w.preshapes[0].origin, w.preshapes[0].voxel)
        assert e.value.status == asicp.ASICP_ERR_INVALID_ARG
        asicp.asicp_run(ctx)                    # the context is still usable
        n = asicp.asicp_best_grasps(ctx, 2, np.zeros(14, np.float32))
        assert n == 2
        del keep
    finally:
        asicp.asicp_destroy(ctx)


def test_planted_duplicates_resolve_to_lowest_index(stream):
    """Exact duplicates of object points in two and in four different screening chunks, with gripper
    points placed on them (squared distance exactly 0): the nearest point must be the lowest index,
    which exercises the two-chunk re-evaluation and the full exact fallback."""
    g = np.random.default_rng(29)
    M = 3000
    R = g.uniform(-0.06, 0.06, (M, 3)).astype(np.float32)
    for i in range(10):
        R[700 + i] = R[i]                  # two chunks
    for i in range(10, 20):
        R[700 + i] = R[1500 + i] = R[2900 + i - 10] = R[i]   # four chunks
    N = 40
    S = np.concatenate([R[:20], R[100:120] + np.float32(1e-3)]).astype(np.float32)
    sdf = -np.ones((8, 8, 8), np.float32)
    for shape in (0, asicp.FWD_SHAPES - 1):       # float32 kernel; tensor-core screening + exact choice
        cfg = asicp.asicp_config_default(P=1, K=1, k_max=1, k_stein=0, conv_tol=-1.0, debug=1, cuda_stream=stream,
                                         fwd_shape=shape)
        ctx = asicp.asicp_create(cfg)
        try:
            asicp.asicp_set_object(ctx, R)
            asicp.asicp_set_gripper_sdf(ctx, 0, S, sdf, np.full(3, -0.1, np.float32), np.float32(0.2 / 7))
            asicp.asicp_set_state(ctx, np.array([[0, 0, 0, 1, 0, 0, 0]], np.float32), 0)
            asicp.asicp_step(ctx, 0)
            st = tl.read_state(ctx, 1, 1, N, M)
        finally:
            asicp.asicp_destroy(ctx)
        idx = st["nn_idx"][0]
        assert np.array_equal(idx[:20], np.arange(20)), shape
        assert np.all(st["nn_d2"][0, :20] == 0.0), shape
        rep = {}
        tl.check_nn(st["s_prime"][0], R, idx, rep)


def test_tensor_core_far_and_tiny_queries(stream):
    """Tensor-core shape on queries its f16 split cannot represent (a particle 40 m away: the scaled
    coordinates leave the f16 range, so the whole cloud is scanned) and on an object cloud of tiny
    extent: indices equal the FP64 argmin over the float32 queries up to near-ties, on both shapes.  The
    two shapes agree exactly on the near particles of the ordinary object; for the far particle (whose
    exact-form float32 distances carry rounding far above the gaps between object points) and the tiny
    object they may pick different near-tie partners: the whole-cloud scan takes the float32 argmin over
    every point, the float32 kernel's screening the float32 argmin over the chunks nearest in exact
    arithmetic."""
    g = np.random.default_rng(31)
    for scale in (1.0, 1e-3):
        M = 1000 + int(scale < 1)                       # a ragged last chunk either way
        R = (g.uniform(-0.05, 0.05, (M, 3)) * scale).astype(np.float32)
        N = 96
        S = (g.uniform(-0.04, 0.04, (N, 3)) * scale).astype(np.float32)
        sdf = -np.ones((8, 8, 8), np.float32)
        theta = np.array([[0.01 * scale, 0, 0, 1, 0, 0, 0], [40.0, 0, 0, 0, 1, 0, 0], [0, 0.02 * scale, 0, 0.5, 0.5, 0.5, 0.5]],
                         np.float32)
        got = []
        for shape in (0, asicp.FWD_SHAPES - 1):
            cfg = asicp.asicp_config_default(P=1, K=3, k_max=1, k_stein=0, conv_tol=-1.0, debug=1, cuda_stream=stream,
                                             fwd_shape=shape)
            ctx = asicp.asicp_create(cfg)
            try:
                asicp.asicp_set_object(ctx, R)
                asicp.asicp_set_gripper_sdf(ctx, 0, S, sdf, np.full(3, -0.1, np.float32), np.float32(0.2 / 7))
                asicp.asicp_set_state(ctx, theta, 0)
                asicp.asicp_step(ctx, 0)
                st = tl.read_state(ctx, 1, 3, N, M)
            finally:
                asicp.asicp_destroy(ctx)
            rep = {}
            tl.check_nn(st["s_prime"].reshape(-1, 3), R, st["nn_idx"].reshape(-1), rep)
            got.append(st["nn_idx"].copy())
        if scale == 1.0:
            assert np.array_equal(got[0][[0, 2]], got[1][[0, 2]])


def test_graph_replay_equals_direct_steps(stream):
    """asicp_run replays a captured CUDA graph of the loop; its poses equal those of the same
    iterations launched one by one with asicp_step, and a second replay repeats them exactly."""
    w = synth.custom_case(P=2, K=16, N=300, M=2500, grid=24, k_max=6, seed=37, k_stein=3)
    import oracle
    th0 = np.tile(oracle.fibonacci_init(w.K, w.objects[0].points.astype(np.float64).mean(0), 0.08),
                  (2, 1)).astype(np.float32)
    ctx = _ctx(w, stream, debug=False)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx, th0)
        a = tl.read_theta(ctx, 32)
        asicp.asicp_run(ctx, th0)
        b = tl.read_theta(ctx, 32)
        asicp.asicp_set_state(ctx, th0, 0)
        for k in range(w.k_max):
            asicp.asicp_step(ctx, k)
        c = tl.read_theta(ctx, 32)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    assert np.array_equal(a, b)
    assert np.array_equal(a, c)


@pytest.mark.parametrize("shape", [0, asicp.FWD_SHAPES - 1])
def test_new_object_of_the_same_size_reuses_the_context(stream, shape):
    """A context that already ran on one object, given a second object with the same point count
    (same layout, same captured loop, whose kernels read the new object's data at replay), gives
    exactly the results of a fresh context on that object; stepping right after the new object
    continues from the kept poses; an object of another size needs new poses before a step."""
    import copy
    import oracle
    w1 = synth.custom_case(P=2, K=16, N=300, M=2500, grid=24, k_max=6, seed=43, k_stein=3)
    w2 = copy.copy(w1)
    w2.objects = [synth.partial_object(2500, 4343)]
    th0 = np.tile(oracle.fibonacci_init(w1.K, np.zeros(3), 0.08), (2, 1)).astype(np.float32)

    def outputs(ctx):
        best = np.zeros(8 * 7, np.float32)
        cost = np.zeros(8, np.float32)
        pre = np.zeros(8, np.int32)
        asicp.asicp_best_grasps(ctx, 8, best, cost, pre)
        return tl.read_theta(ctx, 32), best, cost, pre

    ctx = _ctx(w1, stream, debug=False, fwd_shape=shape)
    try:
        keep = tl.upload(ctx, w1)
        asicp.asicp_run(ctx, th0)
        R2 = torch.from_numpy(np.ascontiguousarray(w2.objects[0].points)).cuda()
        asicp.asicp_set_object(ctx, R2)
        asicp.asicp_run(ctx, th0)
        reused = outputs(ctx)
        asicp.asicp_set_state(ctx, th0, 0)
        asicp.asicp_step(ctx, 0)
        stepped = tl.read_theta(ctx, 32)
        asicp.asicp_set_object(ctx, R2)         # same size: the poses stay set
        asicp.asicp_step(ctx, 1)
        R3 = torch.from_numpy(np.ascontiguousarray(synth.partial_object(2600, 4444).points)).cuda()
        asicp.asicp_set_object(ctx, R3)         # another size: new poses needed
        with pytest.raises(asicp.AsicpError) as e:
            asicp.asicp_step(ctx, 2)
        assert e.value.status == asicp.ASICP_ERR_STATE
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    ctx = _ctx(w2, stream, debug=False, fwd_shape=shape)
    try:
        keep = tl.upload(ctx, w2)
        asicp.asicp_run(ctx, th0)
        fresh = outputs(ctx)
        asicp.asicp_set_state(ctx, th0, 0)
        asicp.asicp_step(ctx, 0)
        fresh_step = tl.read_theta(ctx, 32)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    for a, b in zip(reused, fresh):
        assert np.array_equal(a, b)
    assert np.array_equal(stepped, fresh_step)


def test_kernel_times_from_graph_replays(stream):
    """With profiling on, asicp_run's graph replays report one timed launch per kernel and pass; the
    tensor-core shape adds one exact-choice launch per matching pass."""
    w = synth.custom_case(P=1, K=8, N=128, M=600, grid=16, k_max=3, seed=41)
    for shape in (0, asicp.FWD_SHAPES - 1):
        ctx = _ctx(w, stream, debug=False, profile=True, fwd_shape=shape)
        try:
            keep = tl.upload(ctx, w)
            for _ in range(2):
                asicp.asicp_run(ctx)
            ms, n = asicp.asicp_kernel_times(ctx, reset=True)
            del keep
        finally:
            asicp.asicp_destroy(ctx)
        exact = 2 * (w.k_max + 1) if shape == asicp.FWD_SHAPES - 1 else 0
        assert n == [2 * (w.k_max + 1)] * 4 + [2 * w.k_stein, exact]
        assert all(t > 0 for t, c in zip(ms, n) if c)


def test_kernel_times_of_the_matching_kernel_only(stream):
    """profile = 2 times the forward-matching kernel alone (one launch per pass); the other kernels
    run untimed, and the results equal those of an untimed context."""
    w = synth.custom_case(P=1, K=8, N=128, M=600, grid=16, k_max=3, seed=41)
    shape = asicp.FWD_SHAPES - 1
    out = []
    for prof in (0, 2):
        ctx = _ctx(w, stream, debug=False, profile=prof, fwd_shape=shape)
        try:
            keep = tl.upload(ctx, w)
            for _ in range(2):
                asicp.asicp_run(ctx)
            if prof:
                ms, n = asicp.asicp_kernel_times(ctx, reset=True)
            out.append(tl.read_theta(ctx, w.K))
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    assert n == [2 * (w.k_max + 1), 0, 0, 0, 0, 0]
    assert ms[0] > 0 and ms[1:] == [0.0] * 5
    assert np.array_equal(out[0], out[1])


def _uneven_batch(seed=43):
    """4 objects with uneven point counts and per-(object, preshape) particle counts."""
    g = np.random.default_rng(seed)
    P, N = 2, 256
    pre = synth.make_preshapes(P, N, 24, seed)
    sizes = [900, 2500, 4100, 1500]
    objs = [synth.partial_object(M, seed + 100 * (o + 1)) for o, M in enumerate(sizes)]
    K = g.choice([8, 16, 24], size=(len(sizes), P)).astype(np.int32)
    return pre, objs, K


@pytest.mark.parametrize("shape", [0, asicp.FWD_SHAPES - 1])
def test_batched_objects_match_solo_runs(stream, shape):
    """Objects optimised together (one launch per kernel covering all of them) give bit-identical
    poses, costs and rankings to running each object alone, with the float32 and with the
    tensor-core matching."""
    pre, objs, K = _uneven_batch()
    P, k_max, k_stein = 2, 6, 3

    def make(nobj):
        cfg = asicp.asicp_config_default(P=P, K=8, k_max=k_max, k_stein=k_stein, conv_tol=-1.0, cuda_stream=stream,
                                         n_objects=nobj, fwd_shape=shape)
        return asicp.asicp_create(cfg)

    ctx = make(len(objs))
    try:
        asicp.asicp_set_particle_counts(ctx, K.ravel())
        for o, ob in enumerate(objs):
            asicp.asicp_set_object_at(ctx, o, ob.points)
        for p, ps in enumerate(pre):
            asicp.asicp_set_gripper_sdf(ctx, p, ps.S, ps.sdf, ps.origin, ps.voxel)
        asicp.asicp_run(ctx)
        T = int(K.sum())
        th_b = np.zeros((T, 7), np.float32)
        cost_b = np.zeros(T)
        asicp.asicp_get_state(ctx, theta=th_b, cost=cost_b)
        best_b = []
        for o in range(len(objs)):
            bt = np.zeros(5 * 7, np.float32)
            bc = np.zeros(5, np.float32)
            bp = np.zeros(5, np.int32)
            asicp.asicp_best_grasps_at(ctx, o, 5, bt, bc, bp)
            best_b.append((bt, bc, bp))
    finally:
        asicp.asicp_destroy(ctx)

    first = 0
    for o, ob in enumerate(objs):
        n = int(K[o].sum())
        ctx = make(1)
        try:
            asicp.asicp_set_particle_counts(ctx, K[o])
            asicp.asicp_set_object(ctx, ob.points)
            for p, ps in enumerate(pre):
                asicp.asicp_set_gripper_sdf(ctx, p, ps.S, ps.sdf, ps.origin, ps.voxel)
            asicp.asicp_run(ctx)
            th = np.zeros((n, 7), np.float32)
            cost = np.zeros(n)
            asicp.asicp_get_state(ctx, theta=th, cost=cost)
            bt = np.zeros(5 * 7, np.float32)
            bc = np.zeros(5, np.float32)
            bp = np.zeros(5, np.int32)
            asicp.asicp_best_grasps(ctx, 5, bt, bc, bp)
        finally:
            asicp.asicp_destroy(ctx)
        assert np.array_equal(th, th_b[first:first + n]), f"object {o}: poses differ from the solo run"
        assert np.array_equal(cost, cost_b[first:first + n]), f"object {o}: costs differ from the solo run"
        for a, b in zip((bt, bc, bp), best_b[o]):
            assert np.array_equal(a, b)
        first += n


@pytest.mark.parametrize("shape", [0, asicp.FWD_SHAPES - 1])
def test_batched_step_teacher_forced(stream, shape):
    """One batched SVGD step against the oracle, object by object (uneven sizes and particle counts),
    with the float32 and with the tensor-core matching."""
    pre, objs, K = _uneven_batch(seed=47)
    import oracle
    P, N = 2, 256
    cfg = asicp.asicp_config_default(P=P, K=8, k_max=4, k_stein=2, conv_tol=-1.0, debug=1, cuda_stream=stream,
                                     n_objects=len(objs), fwd_shape=shape)
    ctx = asicp.asicp_create(cfg)
    try:
        asicp.asicp_set_particle_counts(ctx, K.ravel())
        for o, ob in enumerate(objs):
            asicp.asicp_set_object_at(ctx, o, ob.points)
        for p, ps in enumerate(pre):
            asicp.asicp_set_gripper_sdf(ctx, p, ps.S, ps.sdf, ps.origin, ps.voxel)
        T = int(K.sum())
        th0 = []
        for o, ob in enumerate(objs):
            for p in range(P):
                th0.append(oracle.fibonacci_init(int(K[o, p]), ob.points.astype(np.float64).mean(0), 0.06))
        asicp.asicp_set_state(ctx, np.ascontiguousarray(np.concatenate(th0), dtype=np.float32), 0)
        before = tl.read_theta(ctx, T)
        asicp.asicp_step(ctx, 1)
        Mtot = sum(int(K[o].sum()) * len(ob.points) for o, ob in enumerate(objs))
        st = {"theta": np.zeros((T, 7), np.float32), "cost": np.zeros(T), "grad": np.zeros((T, 7)),
              "ncol": np.zeros(T, np.int32), "nn_idx": np.zeros((T, N), np.int32),
              "s_prime": np.zeros((T, N, 3), np.float32), "col_list": np.zeros(Mtot, np.int32),
              "col_nn": np.zeros(Mtot, np.int32)}
        asicp.asicp_get_state(ctx, **st)
    finally:
        asicp.asicp_destroy(ctx)
    rep = {}
    cfirst = 0
    for o, ob in enumerate(objs):
        orc = oracle.Oracle(np.stack([ps.S for ps in pre]), [(ps.sdf, ps.origin, ps.voxel) for ps in pre], ob.points)
        M = len(ob.points)
        first_o = sum(int(K[q].sum()) for q in range(o))
        for pk in range(first_o, first_o + int(K[o].sum())):
            p = next(pp for pp in range(P) if pk < first_o + int(K[o, :pp + 1].sum()))
            th = before[pk].astype(np.float64)
            tl.check_nn(st["s_prime"][pk], orc.R, st["nn_idx"][pk], rep)
            n = int(st["ncol"][pk])
            base = cfirst + (pk - first_o) * M
            lst_g = st["col_list"][base:base + n]
            lst_o, vals = orc.collision_points(p, th)
            if not np.array_equal(lst_g, lst_o):
                diff = np.setxor1d(lst_g, lst_o)
                assert np.all(np.abs(vals[diff]) <= tl.PHI_TOL)
                continue
            if n > 0:
                cost_o, g_o = orc.collision_terms(p, th, lst_g, st["col_nn"][base:base + n])
            else:
                cost_o, g_o = orc.match_terms(p, th, st["nn_idx"][pk])
            assert abs(st["cost"][pk] - cost_o) <= tl.COST_GRAD_REL * abs(cost_o) + tl.COST_ABS
            for blk in (slice(0, 3), slice(3, 7)):
                e = np.linalg.norm(st["grad"][pk, blk] - g_o[blk])
                assert e <= tl.COST_GRAD_REL * np.linalg.norm(g_o[blk]) + tl.GRAD_ABS
        cfirst += int(K[o].sum()) * M
    print("batched step:", rep)


def test_every_forward_shape_gives_the_same_correspondences(stream):
    """Each forward-matching kernel shape (queries per thread x screening chunk) on a ragged case
    (N=700, M=5000: partial query block, partial chunk and tile): identical indices, equal to the
    oracle's; the autotuner picks the shape it timed fastest."""
    w = synth.custom_case(P=2, K=20, N=700, M=5000, grid=24, k_max=3, seed=19)
    P, K, N, Mc = 2, w.K, 700, len(w.objects[0].points)
    orc = tl.make_oracle(w)
    import oracle
    com = orc.R.mean(0)
    theta0 = np.tile(oracle.fibonacci_init(K, com, 0.08), (P, 1)).astype(np.float32)
    got = []
    for v in range(asicp.FWD_SHAPES):
        ctx = _ctx(w, stream, debug=1, fwd_shape=v)
        try:
            keep = tl.upload(ctx, w)
            asicp.asicp_set_state(ctx, theta0, 0)
            before = tl.read_theta(ctx, P * K)
            asicp.asicp_step(ctx, 0)
            st = tl.read_state(ctx, P, K, N, Mc)
            got.append(st["nn_idx"].copy())
            if v == 0:
                tl.check_step(orc, w, before, st, 0, {})
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    for v in range(1, len(got)):
        assert np.array_equal(got[v], got[0]), f"shape {v} differs from shape 0"

    ctx = _ctx(w, stream)
    try:
        keep = tl.upload(ctx, w)
        chosen, ms = asicp.asicp_autotune(ctx)
        assert 0 <= chosen < asicp.FWD_SHAPES
        assert all(t > 0 for t in ms) and ms[chosen] == min(ms)
        del keep
    finally:
        asicp.asicp_destroy(ctx)


def _step_indices(w, stream, theta0, shape, k=0):
    """Correspondences and transformed points of one teacher-forced step with kernel shape `shape`."""
    P, K, N, Mc = len(w.preshapes), w.K, w.preshapes[0].S.shape[0], len(w.objects[0].points)
    ctx = _ctx(w, stream, debug=1, fwd_shape=shape)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_set_state(ctx, theta0, k)
        asicp.asicp_step(ctx, k)
        st = tl.read_state(ctx, P, K, N, Mc)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    return st


def test_tensor_core_matching_equals_float32_matching(stream):
    """The tensor-core kernel (split-f16 screening + exact choice) against the float32 kernel at the
    paper's N and M (3 preshapes x 64 particles, N=2048, M=8192; 1.2e6 queries): identical indices
    except near-ties (|d2 difference| <= 1e-6 relative in float64), and ties broken alike."""
    w = synth.custom_case(P=3, K=64, N=2048, M=8192, grid=32, k_max=2, seed=synth.BASE_SEED + 2)
    import oracle
    com = w.objects[0].points.astype(np.float64).mean(0)
    tc = asicp.FWD_VARIANTS.index("tc-f16x3-m128-n256")
    for radius in (0.15, 0.03):          # far from the object, and fingers in contact
        th = np.tile(oracle.fibonacci_init(w.K, com, radius), (3, 1)).astype(np.float32)
        a = _step_indices(w, stream, th, 0)
        b = _step_indices(w, stream, th, tc)
        assert np.array_equal(a["s_prime"], b["s_prime"])
        diff = np.nonzero(a["nn_idx"] != b["nn_idx"])
        n_diff = len(diff[0])
        print(f"radius {radius}: {n_diff} of {a['nn_idx'].size} indices differ")
        if n_diff:
            R = w.objects[0].points.astype(np.float64)
            sp = a["s_prime"][diff].astype(np.float64)
            da = ((sp - R[a["nn_idx"][diff]]) ** 2).sum(-1)
            db = ((sp - R[b["nn_idx"][diff]]) ** 2).sum(-1)
            rel = np.abs(da - db) / np.maximum(np.minimum(da, db), 1e-300)
            assert rel.max() <= tl.NEAR_TIE_REL, f"non-tie mismatch, relative gap {rel.max():.3e}"
            assert n_diff <= 1e-4 * a["nn_idx"].size
        assert np.allclose(a["cost"], b["cost"], rtol=1e-6, atol=0)


def test_separate_collision_cloud_with_a_table(stream):
    """Matching against the object R, collision test against C = R + a table under the object
    (Section IV-C): poses close enough that fingers reach into the table; teacher-forced steps in
    both phases, every output compared with the oracle built with the same C."""
    import oracle
    w = synth.custom_case(P=2, K=16, N=600, M=3000, grid=32, k_max=8, seed=23, k_stein=3)
    R = w.objects[0].points
    C = np.concatenate([R, synth.table_points(2000, R, seed=5)]).astype(np.float32)
    orc = oracle.Oracle(np.stack([pre.S for pre in w.preshapes]),
                        [(pre.sdf, pre.origin, pre.voxel) for pre in w.preshapes], R, Cc=C, K=w.K)
    P, K, N, Mc = 2, w.K, 600, len(C)
    ctx = _ctx(w, stream)
    rep = {}
    table_hits = 0
    try:
        keep = tl.upload(ctx, w)
        Rt, Ct = torch.from_numpy(R).cuda(), torch.from_numpy(C).cuda()
        asicp.asicp_set_object(ctx, Rt, Ct)
        com = R.astype(np.float64).mean(0)
        theta0 = np.tile(oracle.fibonacci_init(K, com, 0.05), (P, 1)).astype(np.float32)
        asicp.asicp_set_state(ctx, theta0, 0)
        for k in (0, 1, 3, 4, 6):
            asicp.asicp_set_state(ctx, tl.read_theta(ctx, P * K), k)
            before = tl.read_theta(ctx, P * K)
            asicp.asicp_step(ctx, k)
            st = tl.read_state(ctx, P, K, N, Mc)
            tl.check_step(orc, w, before, st, k, rep)
            table_hits += sum(int((st["col_list"][pk, :n] >= len(R)).sum()) for pk, n in enumerate(st["ncol"]))
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    print("table:", rep, "table points in collision:", table_hits)
    assert rep.get("colliding_particles", 0) > 0 and table_hits > 0, "the table is meant to be hit"


def test_quarter_sphere_initialisation_matches_oracle(stream):
    """config.init_mode = 1: the quarter-sphere lattice plus six poses above, per preshape group,
    against the oracle's (float32 poses vs float64)."""
    import oracle
    w = synth.custom_case(P=2, K=40, N=200, M=1000, grid=24, k_max=0, seed=29, k_stein=0)
    ctx = _ctx(w, stream, init_mode=1, k_max=0, k_stein=0)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx)
        th = tl.read_theta(ctx, 2 * w.K)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    ref = oracle.quarter_init(w.K, w.objects[0].points.astype(np.float64).mean(0), 0.15)
    for p in range(2):
        got = th[p * w.K:(p + 1) * w.K].astype(np.float64)
        assert np.allclose(got[:, :3], ref[:, :3], rtol=0, atol=2e-7)
        dots = np.abs((got[:, 3:] * ref[:, 3:]).sum(1))          # q and -q are the same rotation
        assert np.all(dots > 1 - 1e-6)


def test_stein_priors_match_oracle(stream):
    """Gaussian translation prior and von Mises rotation prior in the SVGD drive (Section IV-A):
    teacher-forced SVGD steps against the oracle with the same priors."""
    import ctypes
    import oracle
    w = synth.custom_case(P=2, K=16, N=400, M=2000, grid=24, k_max=6, seed=37, k_stein=6, schedule=1)
    mu = np.array([0.5, 0.5, -0.5, 0.5])
    prior = (0.05, 2.0, mu, w.objects[0].points.astype(np.float64).mean(0))
    orc = tl.make_oracle(w)
    P, K, N, Mc = 2, w.K, 400, len(w.objects[0].points)
    cfg = tl.make_config(w, stream=stream, prior_t_sigma=prior[0], prior_q_kappa=prior[1])
    cfg.prior_q_mean = (ctypes.c_float * 4)(*mu)
    ctx = asicp.asicp_create(cfg)
    rep = {}
    try:
        keep = tl.upload(ctx, w)
        theta0 = np.tile(oracle.fibonacci_init(K, prior[3], 0.1), (P, 1)).astype(np.float32)
        asicp.asicp_set_state(ctx, theta0, 0)
        for k in (0, 2, 4):
            asicp.asicp_set_state(ctx, tl.read_theta(ctx, P * K), k)
            before = tl.read_theta(ctx, P * K)
            asicp.asicp_step(ctx, k)
            st = tl.read_state(ctx, P, K, N, Mc)
            tl.check_step(orc, w, before, st, k, rep, prior=prior)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    print("priors:", rep)


def test_minibatch_ramp_matches_oracle(stream):
    """Table I's mini-batch ramp: iteration k matches against a seeded ascending subset of R (one
    point at k = 0, the whole cloud from 2 k_max / 3 on); the collision test and the CoM keep the
    whole object.  Teacher-forced steps against an oracle built on the same subset."""
    import oracle
    w = synth.custom_case(P=2, K=16, N=400, M=3000, grid=24, k_max=12, seed=41, k_stein=4)
    R = w.objects[0].points
    off, idx = synth.minibatch_ramp(len(R), w.k_max, seed=7)
    com = R.astype(np.float64).mean(0)
    S = np.stack([pre.S for pre in w.preshapes])
    sdfs = [(pre.sdf, pre.origin, pre.voxel) for pre in w.preshapes]
    P, K, N = 2, w.K, 400
    ctx = _ctx(w, stream)
    rep = {}
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_set_minibatch(ctx, off, idx)
        theta0 = np.tile(oracle.fibonacci_init(K, com, 0.08), (P, 1)).astype(np.float32)
        asicp.asicp_set_state(ctx, theta0, 0)
        for k in (0, 1, 5, 9):
            sub = R[idx[off[k]:off[k + 1]]]
            orc = oracle.Oracle(S, sdfs, sub, Cc=R, K=K, com=com)
            asicp.asicp_set_state(ctx, tl.read_theta(ctx, P * K), k)
            before = tl.read_theta(ctx, P * K)
            asicp.asicp_step(ctx, k)
            st = tl.read_state(ctx, P, K, N, len(R))
            assert st["nn_idx"].max() < len(sub)
            tl.check_step(orc, w, before, st, k, rep)
        # switching the mini-batches off restores whole-cloud matching
        asicp.asicp_set_minibatch(ctx, None, None)
        asicp.asicp_step(ctx, 3)
        st = tl.read_state(ctx, P, K, N, len(R))
        assert st["nn_idx"].max() > len(R) // 2
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    print("mini-batch:", rep)


@pytest.mark.slow
def test_paper_scale_free_running_final_poses(stream):
    """The paper-scale problem (3 preshapes x 256 particles, N=2048, M=8192, SDF 64^3, 38 SVGD +
    62 SGD iterations) run free on the GPU in the benchmark's launch configuration (tensor-core
    matching, convergence criterion on), against the oracle run free from the same initial poses.
    Stein couples only the particles of one preshape, so the oracle runs preshape 0 alone (the same
    computation, a third of the CPU time).  Required: every particle without a near-tie decision
    along its oracle trajectory within 1 mm / 1e-3 rad (distribution reported), a median position
    error below 1 um, the same non-colliding particles with costs within 1e-4, and the same best
    particle."""
    import os
    import oracle
    w = synth.paper_scale_case()
    P, K = len(w.preshapes), w.K
    tol = float(np.float32(2e-4))
    com = w.objects[0].points.astype(np.float64).mean(0)
    theta0 = np.tile(oracle.fibonacci_init(K, com, 0.15), (P, 1)).astype(np.float32)
    ctx = _ctx(w, stream, debug=False, fwd_shape=asicp.FWD_SHAPES - 1, conv_tol=2e-4)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx, theta0)
        st = tl.read_state(ctx, P, K, w.preshapes[0].S.shape[0], len(w.objects[0].points), debug=False)
        del keep
    finally:
        asicp.asicp_destroy(ctx)

    pre = w.preshapes[0]
    orc = oracle.Oracle(pre.S[None], [(pre.sdf, pre.origin, pre.voxel)], w.objects[0].points, K=K)
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, g0=w.g0, g1=w.g1,
                         C_cycles=w.C_cycles, p_exp=w.p_exp, N=orc.N, conv_tol=tol)
    ost, traj, near = tl.oracle_free_run(orc, theta0[:K].astype(np.float64)[None], sched,
                                         nthreads=os.cpu_count() or 1, conv_tol=tol)
    th = st["theta"][:K]
    dpos, dang, tie = tl.compare_final_poses(th, ost["theta"][0], orc, traj, near, "paper scale")
    assert np.median(dpos) <= 1e-6
    ncol_g, ncol_o = st["ncol"][:K], ost["ncol"].ravel()
    close = (dpos <= tl.POSE_TOL_M) & (dang <= tl.POSE_TOL_RAD)
    free = (ncol_o == 0) & close
    assert np.array_equal((ncol_g == 0)[close], (ncol_o == 0)[close]), "different non-colliding particles"
    if free.any():
        cg, co = st["cost"][:K][free], ost["cost"].ravel()[free]
        assert np.all(np.abs(cg - co) <= 1e-4 * np.abs(co) + tl.COST_ABS), (cg, co)
    best_g = oracle.select(st["cost"][:K], ncol_g, 1)[0]
    best_o = oracle.select(ost["cost"].ravel(), ncol_o, 1)[0]
    assert best_g == best_o or not (close[best_g] and close[best_o]), (best_g, best_o)


def test_largest_workload_sampled_steps_and_tensor_core_agreement(stream):
    """3 x 1024 particles, N=4096, M=65536 (superquadric partial view), SDF 128^3 -- the maximum
    particle count per preshape and the largest clouds: sampled particles of an SVGD and an SGD step
    against the oracle with both matching shapes, from the initial shell (0.15 m) and from contact
    poses (0.04 m, fingers in the object) -- cost, gradient and SGD-updated pose errors against the
    FP64 oracle reported -- and the tensor-core kernel's correspondences against the float32
    kernel's on every query (identical except near-ties)."""
    import oracle
    w = synth.large_case()
    g = np.random.default_rng(4)
    sample = sorted(g.choice(w.K * 3, 6, replace=False).tolist())
    rep = _teacher_forced_run(w, stream, [0, 7], {}, sample=sample)
    print("largest workload sampled (float32):", rep)
    com = w.objects[0].points.astype(np.float64).mean(0)
    for radius in (0.15, 0.04):
        th0 = np.tile(oracle.fibonacci_init(w.K, com, radius), (3, 1)).astype(np.float32)
        rep = _teacher_forced_run(w, stream, [0, 7], {}, sample=sample, theta0=th0,
                                  fwd_shape=asicp.FWD_SHAPES - 1)
        print(f"largest workload sampled (tensor cores, radius {radius}): error vs the FP64 oracle: "
              f"cost {rep.get('max_cost_rel', 0):.2e} relative, gradient {rep.get('max_grad_rel', 0):.2e} "
              f"relative, SGD-updated pose {rep.get('max_update_abs', 0):.2e} abs;", rep)
        if radius < 0.1:
            assert rep.get("colliding_particles", 0) > 0
    th = np.tile(oracle.fibonacci_init(w.K, com, 0.15), (3, 1)).astype(np.float32)
    a = _step_indices(w, stream, th, 0)
    b = _step_indices(w, stream, th, asicp.FWD_VARIANTS.index("tc-f16x3-m128-n256"))
    diff = np.nonzero(a["nn_idx"] != b["nn_idx"])
    n_diff = len(diff[0])
    print(f"tensor-core vs float32: {n_diff} of {a['nn_idx'].size} indices differ")
    if n_diff:
        R = w.objects[0].points.astype(np.float64)
        sp = a["s_prime"][diff].astype(np.float64)
        da = ((sp - R[a["nn_idx"][diff]]) ** 2).sum(-1)
        db = ((sp - R[b["nn_idx"][diff]]) ** 2).sum(-1)
        assert (np.abs(da - db) / np.maximum(np.minimum(da, db), 1e-300)).max() <= tl.NEAR_TIE_REL
        assert n_diff <= 1e-4 * a["nn_idx"].size


@pytest.mark.slow
def test_largest_workload_free_running_final_poses(stream):
    """The mixed-precision configuration (3 x 1024 particles, N=4096, M=65536, SDF 128^3) run free for
    its 10 parity iterations (4 SVGD + 6 SGD) on the tensor cores, from contact poses (0.06 m),
    against the oracle run free on preshape 0: the final pose and cost errors against FP64 reported,
    every particle without a near-tie decision within 1 mm / 1e-3 rad."""
    import os
    import oracle
    w = synth.large_case()
    P, K = 3, w.K
    com = w.objects[0].points.astype(np.float64).mean(0)
    theta0 = np.tile(oracle.fibonacci_init(K, com, 0.06), (P, 1)).astype(np.float32)
    ctx = _ctx(w, stream, debug=False, fwd_shape=asicp.FWD_SHAPES - 1)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx, theta0)
        st = tl.read_state(ctx, P, K, 4096, 65536, debug=False)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    pre = w.preshapes[0]
    orc = oracle.Oracle(pre.S[None], [(pre.sdf, pre.origin, pre.voxel)], w.objects[0].points, K=K)
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, g0=w.g0, g1=w.g1,
                         C_cycles=w.C_cycles, p_exp=w.p_exp, N=orc.N)
    ost, traj, near = tl.oracle_free_run(orc, theta0[:K].astype(np.float64)[None], sched,
                                         nthreads=os.cpu_count() or 1)
    dpos, dang, tie = tl.compare_final_poses(st["theta"][:K], ost["theta"][0], orc, traj, near, "largest workload")
    close = (dpos <= tl.POSE_TOL_M) & (dang <= tl.POSE_TOL_RAD)
    free = close & (ost["ncol"].ravel() == 0) & (st["ncol"][:K] == 0)
    crel = np.abs(st["cost"][:K][free] - ost["cost"].ravel()[free]) / np.abs(ost["cost"].ravel()[free])
    print(f"largest workload final cost error vs FP64 (non-colliding particles): max {crel.max():.2e}, "
          f"median {np.median(crel):.2e}")
    assert crel.max() <= 1e-4


def test_convergence_freeze_teacher_forced(stream):
    """Table I's convergence criterion (0.02 %) with the default conv_tol on the GPU, teacher-forced
    in the SGD phase against the oracle on the same poses and previous costs: (1) every particle
    frozen with no previous cost: colliding particles are unfrozen and take the collision step
    (Section IV-D), the others keep their poses exactly; (2) previous costs set so that the relative
    change is 0.5x or 2x the criterion, up or down: the freeze decisions, the kept poses and the SGD
    steps of the others equal the oracle's."""
    import oracle
    w = synth.custom_case(P=2, K=16, N=300, M=1500, grid=24, k_max=6, seed=53, k_stein=2)
    tol = float(np.float32(2e-4))            # the GPU compares against the float32 config value
    orc = tl.make_oracle(w)
    P, K, N, Mc = 2, w.K, 300, len(w.objects[0].points)
    com = orc.R.mean(0)
    # preshape 0 close enough for its fingers to reach into the object, preshape 1 farther out
    theta0 = np.concatenate([oracle.fibonacci_init(K, com, 0.05), oracle.fibonacci_init(K, com, 0.12)]).astype(np.float32)
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, g0=w.g0, g1=w.g1,
                         C_cycles=w.C_cycles, p_exp=w.p_exp, N=orc.N, conv_tol=tol)
    ctx = _ctx(w, stream, conv_tol=2e-4)
    rep = {}
    try:
        keep = tl.upload(ctx, w)
        # (1) all frozen, no previous cost
        asicp.asicp_set_state(ctx, theta0, 3)
        before = tl.read_theta(ctx, P * K)
        asicp.asicp_set_convergence(ctx, np.full(P * K, -1.0), np.ones(P * K, np.int32))
        asicp.asicp_step(ctx, 3)
        st = tl.read_state(ctx, P, K, N, Mc)
        tl.check_step(orc, w, before, st, 3, rep)
        ost = orc.new_state(before.astype(np.float64).reshape(P, K, 7))
        ost["frozen"][:] = 1
        orc.step(ost, sched, 3)
        assert np.array_equal(st["frozen"], ost["frozen"].ravel())
        assert np.array_equal(st["frozen"] == 0, st["ncol"] > 0)
        n_col = int((st["ncol"] > 0).sum())
        assert 0 < n_col < P * K, "the case is meant to have colliding and free particles"
        L = st["cost"].copy()
        # (2) relative changes around the criterion
        rel = np.resize([0.5, 2.0, -0.5, -2.0], P * K) * tol
        prev = L / (1.0 + rel)
        asicp.asicp_set_state(ctx, before, 3)
        asicp.asicp_set_convergence(ctx, prev, np.zeros(P * K, np.int32))
        asicp.asicp_step(ctx, 3)
        st = tl.read_state(ctx, P, K, N, Mc)
        tl.check_step(orc, w, before, st, 3, rep)
        ost = orc.new_state(before.astype(np.float64).reshape(P, K, 7))
        ost["prev_cost"][:] = prev.reshape(P, K)
        orc.step(ost, sched, 3)
        assert np.array_equal(st["frozen"], ost["frozen"].ravel())
        expect = (np.abs(rel) < tol) & (st["ncol"] == 0)
        assert np.array_equal(st["frozen"].astype(bool), expect)
        assert expect.sum() > 0 and (~expect).sum() > 0
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    print("convergence freeze:", rep, "colliding:", n_col)


def test_free_running_with_convergence_freeze(stream):
    """15 SVGD + 25 SGD iterations (Table I's split) run free with the default convergence criterion
    on both sides: the same particles end frozen (except near-criterion decisions) and every particle
    without a near-tie decision ends within 1 mm / 1e-3 rad of the oracle.  On these procedural
    shapes the particles of a real preshape end in contact and keep colliding (a collision unfreezes,
    Section IV-D), so preshape 1 is given an SDF that is negative everywhere: its particles converge
    free of collisions and freeze."""
    import oracle
    w = synth.custom_case(P=2, K=24, N=256, M=1024, grid=32, k_max=40, seed=59, k_stein=15)
    w.preshapes[1].sdf = -np.ones_like(w.preshapes[1].sdf)
    tol = float(np.float32(2e-4))
    orc = tl.make_oracle(w)
    P, K = 2, w.K
    theta0 = np.tile(oracle.fibonacci_init(K, orc.R.mean(0), 0.08), (P, 1)).astype(np.float32)
    sched = orc.schedule(k_max=w.k_max, k_stein=w.k_stein, schedule=w.schedule, g0=w.g0, g1=w.g1,
                         C_cycles=w.C_cycles, p_exp=w.p_exp, N=orc.N, conv_tol=tol)
    ost, traj, near = tl.oracle_free_run(orc, theta0.astype(np.float64).reshape(P, K, 7), sched, nthreads=8,
                                         conv_tol=tol)
    ctx = _ctx(w, stream, debug=False, conv_tol=2e-4, fwd_shape=asicp.FWD_SHAPES - 1)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_run(ctx, theta0)
        st = tl.read_state(ctx, P, K, 256, 1024, debug=False)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    frz_o = ost["frozen"].ravel().astype(bool)
    frz_g = st["frozen"].astype(bool)
    dpos, dang, tie = tl.compare_final_poses(st["theta"], ost["theta"], orc, traj, near, "free run with freezing")
    differ = np.nonzero(frz_g != frz_o)[0]
    print(f"frozen: gpu {frz_g.sum()}, oracle {frz_o.sum()} of {P * K}; differing {len(differ)}")
    assert frz_o.sum() > 0, "the run is meant to freeze particles"
    for i in differ:          # a different freeze decision only where a decision was near a tie
        assert near.ravel()[i] or tl.trajectory_margin(orc, traj, i // K, i % K) < tl.FLIP_MARGIN, i


def test_translated_object_matches_oracle_and_keeps_screening_cost(stream):
    """An object cloud far from the coordinate origin (translated by (0.5, 0.3, 0.8) m, as a camera- or
    robot-frame capture would be): teacher-forced SVGD and SGD steps with both matching shapes equal
    the oracle's, and the screening stays as selective as for the centred cloud -- the error windows
    are measured from the object's own frame centre, so the tensor-core screening and exact choice
    take the same time (within 5 %; measured within 0.2 % on GB300) as for the same cloud at the
    origin: the exact choice would rescan far more chunks if the windows grew."""
    import oracle
    shift = np.array([0.5, 0.3, 0.8], np.float32)
    w0 = synth.custom_case(P=1, K=128, N=2048, M=8192, grid=32, k_max=4, seed=61, k_stein=2)
    w1 = synth.custom_case(P=1, K=128, N=2048, M=8192, grid=32, k_max=4, seed=61, k_stein=2)
    w1.objects[0].points = (w0.objects[0].points + shift).astype(np.float32)
    times = []
    for w in (w0, w1):
        orc = tl.make_oracle(w)
        com = orc.R.mean(0)
        th0 = oracle.fibonacci_init(w.K, com, 0.05).astype(np.float32)
        for shape in (0, asicp.FWD_SHAPES - 1):
            rep = {}
            ctx = _ctx(w, stream, fwd_shape=shape)
            try:
                keep = tl.upload(ctx, w)
                asicp.asicp_set_state(ctx, th0, 0)
                for k in (0, 2):
                    asicp.asicp_set_state(ctx, tl.read_theta(ctx, w.K), k)
                    before = tl.read_theta(ctx, w.K)
                    asicp.asicp_step(ctx, k)
                    st = tl.read_state(ctx, 1, w.K, 2048, 8192)
                    sample = list(range(0, w.K, 4))
                    tl.check_step(orc, w, before, st, k, rep, sample=sample)
                del keep
            finally:
                asicp.asicp_destroy(ctx)
            print("translated" if w is w1 else "centred", "shape", shape, rep)
        ctx = _ctx(w, stream, debug=False, profile=True, fwd_shape=asicp.FWD_SHAPES - 1)
        try:
            keep = tl.upload(ctx, w)
            asicp.asicp_set_state(ctx, th0, 0)
            for _ in range(3):
                asicp.asicp_step(ctx, 0)
            asicp.asicp_kernel_times(ctx, reset=True)
            for _ in range(10):
                asicp.asicp_step(ctx, 0)
            ms, n = asicp.asicp_kernel_times(ctx, reset=True)
            times.append((ms[0] + ms[5]) / n[0])
            del keep
        finally:
            asicp.asicp_destroy(ctx)
    print(f"matching per launch: centred {times[0]:.4f} ms, translated {times[1]:.4f} ms")
    assert times[1] <= 1.05 * times[0]


def test_bounded_wait_timeout_is_reported_and_the_context_recovers(stream):
    """Every device wait of the library is bounded.  With the float32 matching kernel's first copy
    wait made on an mbarrier that nothing arrives at (a 1000-cycle limit), every CTA's wait expires:
    the kernel drains its copies and returns, the later kernels of the pass skip their work, the
    next read-back returns TIMEOUT naming the expired wait, and with normal waits restored the same
    context computes the step exactly as a fresh context does."""
    import oracle
    w = synth.custom_case(P=2, K=16, N=300, M=5000, grid=24, k_max=4, seed=67, k_stein=2)
    P, K, N, Mc = 2, w.K, 300, 5000
    th0 = np.tile(oracle.fibonacci_init(K, w.objects[0].points.astype(np.float64).mean(0), 0.06),
                  (P, 1)).astype(np.float32)
    ctx = _ctx(w, stream, fwd_shape=0)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_set_state(ctx, th0, 0)
        asicp.asicp_test_expire_waits(ctx, True)
        asicp.asicp_step(ctx, 0)
        with pytest.raises(asicp.AsicpError) as e:
            tl.read_state(ctx, P, K, N, Mc)
        assert e.value.status == asicp.ASICP_ERR_TIMEOUT
        assert "wait expired" in asicp.asicp_last_error(ctx)
        asicp.asicp_test_expire_waits(ctx, False)
        asicp.asicp_set_state(ctx, th0, 0)
        asicp.asicp_step(ctx, 0)
        got = tl.read_state(ctx, P, K, N, Mc)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    ctx = _ctx(w, stream, fwd_shape=0)
    try:
        keep = tl.upload(ctx, w)
        asicp.asicp_set_state(ctx, th0, 0)
        asicp.asicp_step(ctx, 0)
        ref = tl.read_state(ctx, P, K, N, Mc)
        del keep
    finally:
        asicp.asicp_destroy(ctx)
    for key in ("theta", "cost", "grad", "ncol", "nn_idx"):
        assert np.array_equal(got[key], ref[key]), key
