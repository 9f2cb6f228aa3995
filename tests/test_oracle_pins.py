"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (scipy rotations, k-d tree, grid interpolation, sorting), a closed
form, an invariant, a special case that reduces to a textbook method
(Kabsch/Horn for Eq. 2, SGD for SVGD with one particle), or brute force on
tiny inputs.  A plausible slip anywhere in the oracle (a dropped term, a wrong
sign or index, a transposed operand) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from paper_2412_08346_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_quat(g):
    q = g.normal(size=4)
    return q / np.linalg.norm(q)


def tangent_dirs(q):
    """Orthonormal basis of the tangent space of S^3 at q."""
    m = np.eye(4) - np.outer(q, q)
    u, s, _ = np.linalg.svd(m)
    return u[:, :3].T


# ------------------------------------------------------------------ rotation
def test_rotation_matches_scipy(oracle_mod):
    g = np.random.default_rng(1)
    for _ in range(50):
        q = rand_quat(g)
        ref = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()   # scipy: (x, y, z, w)
        assert np.allclose(oracle_mod.rotation(q), ref, atol=1e-14)


def test_rotation_known_axes_and_double_cover(oracle_mod):
    c = math.sqrt(0.5)
    # 90 degrees about x maps y -> z, about y maps z -> x, about z maps x -> y
    assert np.allclose(oracle_mod.rotation([c, c, 0, 0]) @ [0, 1, 0], [0, 0, 1], atol=1e-15)
    assert np.allclose(oracle_mod.rotation([c, 0, c, 0]) @ [0, 0, 1], [1, 0, 0], atol=1e-15)
    assert np.allclose(oracle_mod.rotation([c, 0, 0, c]) @ [1, 0, 0], [0, 1, 0], atol=1e-15)
    g = np.random.default_rng(2)
    for _ in range(20):
        q = rand_quat(g)
        R = oracle_mod.rotation(q)
        assert np.abs(R.T @ R - np.eye(3)).max() < 1e-15 * 10
        assert abs(np.linalg.det(R) - 1) < 1e-14
        assert np.array_equal(R, oracle_mod.rotation(-q))


def test_rotation_jacobian_finite_difference(oracle_mod):
    """dR(q)s/dq of Eqs. 5/17 against central differences of the (scipy-pinned) rotation."""
    g = np.random.default_rng(3)
    for _ in range(20):
        q = rand_quat(g)
        s = g.normal(size=3) * 0.05
        J = oracle_mod.rot_jacobian(q, s)
        h = 1e-6
        for k in range(4):
            dq = np.zeros(4)
            dq[k] = h
            # the homogeneous form is a quadratic polynomial in q: central differences are exact up to rounding
            fd = (oracle_mod.rotation(q + dq) @ s - oracle_mod.rotation(q - dq) @ s) / (2 * h)
            assert np.allclose(J[:, k], fd, atol=1e-10)


# ------------------------------------------------------------------ matching (Eq. 1)
def test_nn_matches_kdtree(oracle_mod):
    g = np.random.default_rng(4)
    Q = g.uniform(-0.1, 0.1, (300, 3))
    Rf = g.uniform(-0.1, 0.1, (700, 3))
    idx, d2 = oracle_mod.nn(Q, Rf)
    dist, kidx = cKDTree(Rf).query(Q)
    assert np.array_equal(idx, kidx)
    assert np.allclose(d2, dist ** 2, rtol=1e-12)


def test_nn_planted_ties_go_to_lowest_index(oracle_mod):
    # references placed symmetrically around each query: exact ties in float64
    Q = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0]])
    Rf = np.array([[5.0, 0, 0], [0.5, 0, 0], [-0.5, 0, 0], [0, 0.5, 0], [1.0, 1.25, 1.0], [1.0, 0.75, 1.0]])
    idx, d2 = oracle_mod.nn(Q, Rf)
    assert list(idx) == [1, 4]
    assert np.array_equal(d2, [0.25, 0.0625])


def test_nn_agrees_with_full_sort(oracle_mod):
    g = np.random.default_rng(5)
    Q = g.integers(-3, 4, (200, 3)).astype(float)      # integer lattice: many exact ties
    Rf = g.integers(-3, 4, (50, 3)).astype(float)
    idx, _ = oracle_mod.nn(Q, Rf)
    for i in range(len(Q)):
        d = ((Rf - Q[i]) ** 2).sum(1)
        order = np.lexsort((np.arange(len(Rf)), d))       # by distance, then index
        assert idx[i] == order[0]


# ------------------------------------------------------------------ SDF lookup (Eq. 12)
def test_trilinear_matches_scipy_and_nodes(oracle_mod):
    g = np.random.default_rng(6)
    grid = g.normal(size=(5, 6, 7))            # [z, y, x]
    origin = np.array([-0.3, 0.1, 0.2])
    voxel = 0.05
    axes = [origin[a] + voxel * np.arange(n) for a, n in enumerate((7, 6, 5))]
    interp = RegularGridInterpolator((axes[2], axes[1], axes[0]), grid)
    for _ in range(200):
        x = np.array([g.uniform(axes[a][0], axes[a][-1]) for a in range(3)])
        v, inside = oracle_mod.trilinear(grid, origin, voxel, x)
        assert inside
        assert abs(v - interp([x[2], x[1], x[0]])[0]) < 1e-12
    # at nodes, including the far corner, the value is the node value
    for (iz, iy, ix) in [(0, 0, 0), (4, 5, 6), (2, 3, 1), (4, 0, 6)]:
        # a hair inside the node box so the far faces do not round outside it
        node = np.array([ix, iy, iz], dtype=float)
        x = origin + voxel * (node + 1e-12 * (np.array([3.0, 2.5, 2.0]) - node))
        v, inside = oracle_mod.trilinear(grid, origin, voxel, x)
        assert inside and abs(v - grid[iz, iy, ix]) < 1e-9
    v, inside = oracle_mod.trilinear(grid, origin, voxel, origin - 1e-9)
    assert not inside


def test_trilinear_exact_on_linear_field_and_sphere_error(oracle_mod):
    n = 17
    voxel = 0.2 / (n - 1)
    origin = np.full(3, -0.1)
    ax = origin[0] + voxel * np.arange(n)
    zz, yy, xx = np.meshgrid(ax, ax, ax, indexing="ij")
    a = np.array([0.3, -1.2, 0.7])
    lin = a[0] * xx + a[1] * yy + a[2] * zz + 0.05
    sph = 0.06 - np.sqrt(xx ** 2 + yy ** 2 + zz ** 2)
    g = np.random.default_rng(7)
    for _ in range(200):
        x = g.uniform(-0.099, 0.099, 3)
        v, _ = oracle_mod.trilinear(lin, origin, voxel, x)
        assert abs(v - (a @ x + 0.05)) < 1e-13
        v, _ = oracle_mod.trilinear(sph, origin, voxel, x)
        r = np.linalg.norm(x)
        if r > 0.03:   # smooth region: interpolation error of a C2 field is O(voxel^2 * curvature)
            assert abs(v - (0.06 - r)) <= 3 * voxel ** 2 / (2 * (r - 0.5 * math.sqrt(3) * voxel))


# ------------------------------------------------------------------ match cost and gradient
def _tiny_problem(oracle_mod, g, N=20, M=60, w_com=1.0, K=1, scale=0.05):
    S = g.uniform(-scale, scale, (1, N, 3))
    Rf = g.uniform(-scale, scale, (M, 3)) + np.array([0.0, 0.0, 0.2])
    grid = -np.ones((4, 4, 4))          # SDF everywhere negative: never colliding
    return oracle_mod.Oracle(S, [(grid, np.full(3, -0.1), 0.2 / 3)], Rf, K=K, w_com=w_com)


def test_match_gradient_is_half_the_cost_derivative(oracle_mod):
    """Eqs. 16/17 against central differences of the cost they belong to (with fixed pairs)."""
    g = np.random.default_rng(8)
    orc = _tiny_problem(oracle_mod, g)
    for trial in range(10):
        q = rand_quat(g)
        th = np.concatenate([g.uniform(-0.05, 0.05, 3) + [0, 0, 0.2], q])
        L, gr, idx = orc.match_cost_grad(0, th)
        h = 1e-7
        for a in range(3):
            tp, tm = th.copy(), th.copy()
            tp[a] += h
            tm[a] -= h
            (Lp, _, ip), (Lm, _, im) = orc.match_cost_grad(0, tp), orc.match_cost_grad(0, tm)
            assert np.array_equal(ip, idx) and np.array_equal(im, idx)
            assert abs((Lp - Lm) / (2 * h) - 2 * gr[a]) <= 1e-6 * max(1.0, abs(2 * gr[a]))
        assert abs(gr[3:] @ q) < 1e-15          # projected onto the tangent space
        for d in tangent_dirs(q):
            qp, qm = q + h * d, q - h * d
            tp = np.concatenate([th[:3], qp / np.linalg.norm(qp)])
            tm = np.concatenate([th[:3], qm / np.linalg.norm(qm)])
            (Lp, _, ip), (Lm, _, im) = orc.match_cost_grad(0, tp), orc.match_cost_grad(0, tm)
            assert np.array_equal(ip, idx) and np.array_equal(im, idx)
            assert abs((Lp - Lm) / (2 * h) - 2 * gr[3:] @ d) <= 1e-6 * max(1e-3, abs(2 * gr[3:] @ d))


def test_match_cost_brute_force_definition(oracle_mod):
    g = np.random.default_rng(9)
    orc = _tiny_problem(oracle_mod, g, w_com=0.7)
    q = rand_quat(g)
    th = np.concatenate([[0.01, -0.02, 0.18], q])
    L, gr, idx = orc.match_cost_grad(0, th)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sp = orc.S[0] @ R.T + th[:3]
    d = ((Sp[:, None, :] - orc.R[None, :, :]) ** 2).sum(-1)
    assert np.array_equal(idx, d.argmin(1))
    tcp, com = orc.S[0].mean(0), orc.R.mean(0)
    ec = R @ tcp + th[:3] - com
    assert abs(L - (d.min(1).sum() + 0.7 * ec @ ec) / orc.N) < 1e-15
    e = Sp - orc.R[idx]
    assert np.allclose(gr[:3], (e.sum(0) + 0.7 * ec) / orc.N, atol=1e-16)


def test_kabsch_optimum_is_stationary(oracle_mod):
    """Eq. 2 solved in closed form (Kabsch/Horn, via SVD): the gradient of Eqs. 4-5 vanishes there."""
    g = np.random.default_rng(10)
    N = 25
    S = g.uniform(-0.05, 0.05, (N, 3))
    R_true = Rotation.random(random_state=11).as_matrix()
    t_true = np.array([0.02, -0.01, 0.3])
    obj = S @ R_true.T + t_true + g.normal(0, 1e-4, (N, 3))   # noisy: optimum has residual
    # Kabsch with pairs i <-> i
    cs, co = S.mean(0), obj.mean(0)
    H = (S - cs).T @ (obj - co)
    U, _, Vt = np.linalg.svd(H)
    D = np.diag([1, 1, np.sign(np.linalg.det(Vt.T @ U.T))])
    Rk = Vt.T @ D @ U.T
    tk = co - Rk @ cs
    xyzw = Rotation.from_matrix(Rk).as_quat()
    q = np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]])
    grid = -np.ones((4, 4, 4))
    orc = oracle_mod.Oracle(S[None], [(grid, np.full(3, -0.1), 0.1)], obj, w_com=0.0)
    L, gr, idx = orc.match_cost_grad(0, np.concatenate([tk, q]))
    assert np.array_equal(idx, np.arange(N))       # the pairing is the identity at the optimum
    assert np.abs(gr).max() < 1e-13
    assert L > 1e-9
    # moving away from the optimum makes the gradient non-zero and the cost larger
    L2, gr2, _ = orc.match_cost_grad(0, np.concatenate([tk + [1e-3, 0, 0], q]))
    assert L2 > L and abs(gr2[0] - 1e-3) < 1e-12


def test_sgd_icp_recovers_known_rigid_transform(oracle_mod):
    """SGD-ICP (Eq. 3, eta = 1, A = I) on a tiny cloud converges to the transform that made the object."""
    g = np.random.default_rng(12)
    N = 20
    S = g.uniform(-0.5, 0.5, (N, 3))
    R_true = Rotation.from_rotvec([0.3, -0.2, 0.1]).as_matrix()
    t_true = np.array([0.1, 0.2, -0.1])
    obj = S @ R_true.T + t_true
    xyzw = Rotation.from_matrix(R_true).as_quat()
    q_true = np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]])
    grid = -np.ones((4, 4, 4))
    orc = oracle_mod.Oracle(S[None], [(grid, np.full(3, -5.0), 10.0 / 3)], obj, K=1, w_com=0.0)
    q0 = q_true + np.array([0.0, 0.02, -0.01, 0.015])
    th0 = np.concatenate([t_true + [0.03, -0.02, 0.01], q0 / np.linalg.norm(q0)])
    sched = orc.schedule(k_max=80, k_stein=0, N=N)
    st = orc.new_state(th0[None, None])
    for k in range(80):
        orc.step(st, sched, k)
    th = st["theta"][0, 0]
    assert np.abs(th[:3] - t_true).max() < 1e-6
    assert min(np.abs(th[3:] - q_true).max(), np.abs(th[3:] + q_true).max()) < 1e-6


def test_pure_translation_step_is_mean_residual(oracle_mod):
    """With identity rotation and w_com = 0, one SGD step moves t by minus the mean residual."""
    g = np.random.default_rng(13)
    orc = _tiny_problem(oracle_mod, g, w_com=0.0)
    th = np.array([0.0, 0.0, 0.19, 1.0, 0.0, 0.0, 0.0])
    L, gr, idx = orc.match_cost_grad(0, th)
    e = orc.S[0] + th[:3] - orc.R[idx]
    st = orc.new_state(th[None, None])
    orc.step(st, orc.schedule(k_max=1, k_stein=0, N=orc.N), 0)
    assert np.allclose(st["theta"][0, 0, :3], th[:3] - e.mean(0), atol=1e-15)


# ------------------------------------------------------------------ collision (Eqs. 12, 18)
def _palm_problem(oracle_mod, pts):
    sdf, origin, voxel = synth.sdf_grid(0.0, 41)
    S = synth.gripper_contact_cloud(64, 0.0, 3).astype(np.float64)
    return oracle_mod.Oracle(S[None], [(sdf, origin, voxel)], np.asarray(pts, dtype=np.float64)), S


def test_collision_single_point_in_palm(oracle_mod):
    # gripper at the origin with identity rotation: the object point (1, 1, -5) mm sits inside the palm plate
    pts = [[0.001, 0.001, -0.005], [0.0, 0.0, 0.05], [0.09, 0.09, 0.09], [0.5, 0.0, 0.0]]
    orc, S = _palm_problem(oracle_mod, pts)
    th = np.array([0, 0, 0, 1.0, 0, 0, 0])
    lst, vals = orc.collision_points(0, th)
    assert list(lst) == [0]
    assert abs(vals[0] - 0.005) < 1e-3          # 5 mm deep: 5 mm from the palm's top and bottom faces
    assert vals[1] < 0 and vals[2] < 0 and vals[3] == -np.inf
    L, gr, nn_ = orc.collision_cost_grad(0, th, lst)
    d = ((S - np.asarray(pts[0])) ** 2).sum(1)
    assert nn_[0] == d.argmin()
    assert abs(L - d.min()) < 1e-15
    assert np.allclose(gr[:3], S[d.argmin()] - pts[0], atol=1e-16)


def test_collision_threshold_is_strictly_inside(oracle_mod):
    """Half a millimetre above the palm's top face is free, half a millimetre below collides."""
    pts = [[0.002, 0.003, 0.0005], [0.002, 0.003, -0.0005], [0.002, 0.003, 0.003]]
    orc, _ = _palm_problem(oracle_mod, pts)
    lst, vals = orc.collision_points(0, np.array([0, 0, 0, 1.0, 0, 0, 0]))
    assert list(lst) == [1]
    # the palm face is the grid plane z = 0: the interpolated SDF there is linear in z
    assert abs(vals[0] + 0.0005) < 1e-8 and abs(vals[1] - 0.0005) < 1e-8   # float32 node values


def test_collision_points_follow_the_pose(oracle_mod):
    """c' = R^T (c - t): a point placed inside the palm of a moved/rotated gripper collides."""
    g = np.random.default_rng(14)
    q = rand_quat(g)
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    t = np.array([0.03, -0.02, 0.05])
    inside_local = np.array([0.01, -0.02, -0.004])     # inside the palm plate
    outside_local = np.array([0.0, 0.0, 0.03])         # between the fingers
    pts = [R @ outside_local + t, R @ inside_local + t]
    orc, _ = _palm_problem(oracle_mod, pts)
    lst, vals = orc.collision_points(0, np.concatenate([t, q]))
    assert list(lst) == [1]
    assert abs(vals[1] - synth.gripper_sdf_value(inside_local[None], 0.0)[0]) < 2e-3


def test_collision_gradient_finite_difference(oracle_mod):
    pts = [[0.001, 0.001, -0.005], [0.02, -0.01, -0.003], [0.0, 0.0, 0.05]]
    orc, S = _palm_problem(oracle_mod, pts)
    g = np.random.default_rng(15)
    q = rand_quat(g) * 0.05 + np.array([1.0, 0, 0, 0])
    q /= np.linalg.norm(q)
    th = np.concatenate([[0.001, 0.0, 0.0], q])
    lst, _ = orc.collision_points(0, th)
    assert len(lst) >= 1
    L, gr, nn_ = orc.collision_cost_grad(0, th, lst)
    h = 1e-7
    for a in range(3):
        tp, tm = th.copy(), th.copy()
        tp[a] += h
        tm[a] -= h
        Lp, _, np_ = orc.collision_cost_grad(0, tp, lst)
        Lm, _, nm = orc.collision_cost_grad(0, tm, lst)
        assert np.array_equal(np_, nn_) and np.array_equal(nm, nn_)
        assert abs((Lp - Lm) / (2 * h) - 2 * gr[a]) < 1e-7
    for d in tangent_dirs(q):
        qp, qm = q + h * d, q - h * d
        Lp, _, _ = orc.collision_cost_grad(0, np.concatenate([th[:3], qp / np.linalg.norm(qp)]), lst)
        Lm, _, _ = orc.collision_cost_grad(0, np.concatenate([th[:3], qm / np.linalg.norm(qm)]), lst)
        assert abs((Lp - Lm) / (2 * h) - 2 * gr[3:] @ d) < 1e-7


def test_collision_replaces_match_gradient_in_step(oracle_mod):
    pts = [[0.001, 0.001, -0.005], [0.0, 0.0, 0.05]]
    orc, S = _palm_problem(oracle_mod, pts)
    th = np.array([0, 0, 0, 1.0, 0, 0, 0])
    st = orc.new_state(th[None, None])
    orc.step(st, orc.schedule(k_max=1, k_stein=0, N=orc.N), 0)
    lst, _ = orc.collision_points(0, th)
    Lc, gc, _ = orc.collision_cost_grad(0, th, lst)
    assert st["ncol"][0, 0] == 1
    assert st["cost"][0, 0] == Lc and np.array_equal(st["grad"][0, 0], gc)


# ------------------------------------------------------------------ annealing and Stein (Eqs. 6-11)
def test_annealing_schedule_closed_form(oracle_mod):
    with open(os.path.join(GOLDEN, "table1_parameters.json")) as f:
        t1 = json.load(f)
    C, p = t1["annealing_cycles_C"], t1["annealing_exponent_p"]
    for k in range(100):
        period = 100 / C
        assert oracle_mod.gamma(k, 100, 0, C, p) == pytest.approx(((k % period) / period) ** p, abs=1e-15)
    assert oracle_mod.gamma(0, 100) == 0.0
    assert oracle_mod.gamma(10, 100) == pytest.approx(0.25)
    assert oracle_mod.gamma(20, 100) == 0.0
    assert oracle_mod.gamma(0, 50, 1) == pytest.approx(0.1)
    assert oracle_mod.gamma(49, 50, 1) == pytest.approx(1.0)


def test_bandwidth_median_heuristic(oracle_mod):
    g = np.random.default_rng(16)
    for K in (2, 3, 7, 32):
        th = np.concatenate([g.normal(size=(K, 3)) * 0.1, np.tile([1.0, 0, 0, 0], (K, 1))], 1)
        d = np.sort([((th[i, :3] - th[j, :3]) ** 2).sum() for i in range(K) for j in range(i + 1, K)])
        med = d[(len(d) - 1) // 2]
        assert oracle_mod.bandwidth(th) == pytest.approx(med / math.log(K), rel=1e-14)
    assert oracle_mod.bandwidth(np.zeros((1, 7))) == 1.0
    assert oracle_mod.bandwidth(np.zeros((4, 7))) == 1e-12
    assert oracle_mod.bandwidth(np.zeros((4, 7)), 1, 0.3) == 0.3


def test_stein_two_particles_repulsion_closed_form(oracle_mod):
    """K = 2, gamma = 0: only the RBF repulsion remains, phi_1 = (1/2)(2/h)(t1 - t2) exp(-|t1-t2|^2/h)."""
    t1, t2 = np.array([0.1, 0.0, 0.02]), np.array([0.0, 0.05, 0.0])
    q1 = np.array([1.0, 0, 0, 0])
    q2 = np.array([0.8, 0.6, 0, 0])
    th = np.array([np.concatenate([t1, q1]), np.concatenate([t2, q2])])
    grad = np.random.default_rng(17).normal(size=(2, 7))
    h = oracle_mod.bandwidth(th)
    d2 = ((t1 - t2) ** 2).sum()
    assert h == pytest.approx(d2 / math.log(2))
    phi = oracle_mod.stein_direction(th, grad, 100, 0.0, h)
    # exp(-d2/h) = exp(-ln 2) = 1/2
    assert np.allclose(phi[0, :3], 0.5 * (2 / h) * (t1 - t2) * 0.5, atol=1e-15)
    assert np.allclose(phi[1, :3], 0.5 * (2 / h) * (t2 - t1) * 0.5, atol=1e-15)
    # the rotational repulsion of the dot-product kernel is radial: projected away
    assert np.abs(phi[:, 3:]).max() < 1e-16


def test_single_particle_svgd_step_equals_sgd_step(oracle_mod):
    """K = 1, gamma = 1, eta_svgd = 1/N: the Stein update (Eq. 7/8) is exactly the SGD-ICP update (Eq. 3)."""
    g = np.random.default_rng(18)
    orc = _tiny_problem(oracle_mod, g, K=1)
    q = rand_quat(g)
    th = np.concatenate([[0.01, 0.0, 0.2], q])
    a = orc.new_state(th[None, None])
    b = orc.new_state(th[None, None])
    orc.step(a, orc.schedule(k_max=2, k_stein=2, schedule=1, g0=1.0, g1=1.0, N=orc.N), 0)
    orc.step(b, orc.schedule(k_max=2, k_stein=0, N=orc.N), 0)
    assert np.allclose(a["theta"], b["theta"], atol=1e-15, rtol=0)
    assert np.allclose(a["phi"][0, 0], -orc.N * b["grad"][0, 0], rtol=1e-12, atol=1e-17)


def test_stein_direction_respects_quaternion_double_cover(oracle_mod):
    """q and -q are one rotation, and the gradient at -q is minus the gradient at q: writing a
    particle either way must not change any particle's Stein direction (the abs of Eq. 10)."""
    g = np.random.default_rng(20)
    K = 5
    th = np.concatenate([g.normal(size=(K, 3)) * 0.03, np.array([rand_quat(g) for _ in range(K)])], 1)
    grad = g.normal(size=(K, 7))
    for i in range(K):
        grad[i, 3:] -= (grad[i, 3:] @ th[i, 3:]) * th[i, 3:]
    h = oracle_mod.bandwidth(th)
    phi = oracle_mod.stein_direction(th, grad, 50, 0.7, h)
    th2, grad2 = th.copy(), grad.copy()
    th2[1, 3:] *= -1
    grad2[1, 3:] *= -1
    phi2 = oracle_mod.stein_direction(th2, grad2, 50, 0.7, h)
    for i in range(K):
        sgn = -1.0 if i == 1 else 1.0
        assert np.allclose(phi2[i, :3], phi[i, :3], atol=1e-15)
        assert np.allclose(phi2[i, 3:], sgn * phi[i, 3:], atol=1e-15)


def test_stein_drive_is_kernel_weighted_mean_gradient(oracle_mod):
    """Far-apart particles (kernel ~ 0 between them) with equal rotations: each is driven by its own gradient / K."""
    th = np.array([[0, 0, 0, 1.0, 0, 0, 0], [100.0, 0, 0, 1.0, 0, 0, 0]])
    grad = np.array([[1.0, 2, 3, 0, 0.1, 0.2, 0.3], [-1.0, 0, 1, 0, 0.3, 0.2, 0.1]])
    phi = oracle_mod.stein_direction(th, grad, 10, 0.5, 1.0)
    assert np.allclose(phi[0, :3], -0.5 * 10 * grad[0, :3] / 2, atol=1e-15)
    # both rotations equal: the rotation kernel is 1 for every pair, the drive is the mean of both
    assert np.allclose(phi[0, 3:], -0.5 * 10 * (grad[0, 3:] + grad[1, 3:]) / 2, atol=1e-15)


# ------------------------------------------------------------------ whole iterations
def _moved(oracle_mod, Rg, tg, th):
    out = th.copy()
    xyzw = Rotation.from_matrix(Rg).as_quat()
    qg = np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]])
    for i in range(len(th)):
        out[i, :3] = Rg @ th[i, :3] + tg
        w1, v1 = qg[0], qg[1:]
        w2, v2 = th[i, 3], th[i, 4:]
        out[i, 3] = w1 * w2 - v1 @ v2
        out[i, 4:] = w1 * v2 + w2 * v1 + np.cross(v1, v2)
    return out


def test_whole_iteration_is_rigid_motion_equivariant(oracle_mod):
    """Moving object and particles by one rigid motion moves every result of a step the same way."""
    w = synth.custom_case(P=1, K=6, N=48, M=96, grid=21, k_max=6, seed=99)
    pre = w.preshapes[0]
    R0 = w.objects[0].points.astype(np.float64)
    Rg = Rotation.from_rotvec([0.4, -0.7, 0.2]).as_matrix()
    tg = np.array([0.3, -0.1, 0.05])
    com = R0.mean(0)
    th0 = oracle_mod.fibonacci_init(6, com, 0.06)
    sdfs = [(pre.sdf, pre.origin, pre.voxel)]
    A = oracle_mod.Oracle(pre.S[None], sdfs, R0, K=6)
    B = oracle_mod.Oracle(pre.S[None], sdfs, R0 @ Rg.T + tg, K=6)
    sched = A.schedule(k_max=6, k_stein=3, N=48)
    sa = A.new_state(th0[None])
    sb = B.new_state(_moved(oracle_mod, Rg, tg, th0)[None])
    any_col = 0
    for k in range(6):
        A.step(sa, sched, k)
        B.step(sb, sched, k)
        any_col += sa["ncol"].sum()
        assert np.array_equal(sa["ncol"], sb["ncol"])
        assert np.allclose(sa["cost"], sb["cost"], rtol=1e-9, atol=1e-15)
        assert np.allclose(_moved(oracle_mod, Rg, tg, sa["theta"][0]), sb["theta"][0], atol=1e-9)


def test_fibonacci_initialisation_closed_form(oracle_mod):
    K, com, rad = 37, np.array([0.01, -0.02, 0.03]), 0.15
    th = oracle_mod.fibonacci_init(K, com, rad)
    ga = math.pi * (3 - math.sqrt(5))
    for j in range(K):
        u = (th[j, :3] - com) / rad
        assert abs(np.linalg.norm(u) - 1) < 1e-14
        assert abs(u[2] - (1 - (2 * j + 1) / K)) < 1e-14
        assert abs(math.atan2(u[1], u[0]) - math.remainder(j * ga, 2 * math.pi)) < 1e-9
        q = th[j, 3:]
        assert abs(np.linalg.norm(q) - 1) < 1e-14 and q[0] >= 0
        R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        assert np.allclose(R @ [0, 0, 1], -u, atol=1e-14)      # approach axis points at the object
        assert abs(q[3]) < 1e-15                                # minimal rotation: axis in the xy plane


def test_selection_order(oracle_mod):
    g = np.random.default_rng(19)
    cost = g.uniform(0, 1, 40)
    cost[5] = cost[9]                      # planted tie: lower index first
    ncol = (g.uniform(0, 1, 40) < 0.3).astype(np.int32)
    order = oracle_mod.select(cost, ncol, 40)
    ref = np.lexsort((np.arange(40), cost, ncol > 0))
    assert np.array_equal(order, ref)


def test_table1_golden_parameters_are_the_defaults(oracle_mod):
    with open(os.path.join(GOLDEN, "table1_parameters.json")) as f:
        t1 = json.load(f)
    assert t1["sgd_learning_rate"] == 1.0
    assert t1["svgd_iterations"] / (t1["svgd_iterations"] + t1["sgd_iterations"]) == 0.375
    assert synth.k_stein_for(40) == t1["svgd_iterations"]
    assert synth.k_stein_for(100) == 38


def test_quarter_sphere_initialisation():
    """Quarter-sphere Fibonacci poses face the CoM from z >= 0, x >= 0 at the given radius, the
    last six sit directly above with the approach axis pointing down, yawed 60 degrees apart."""
    import oracle
    com = np.array([0.01, -0.02, 0.03])
    K, r = 40, 0.15
    th = oracle.quarter_init(K, com, r)
    t, q = th[:, :3] - com, th[:, 3:]
    assert np.allclose(np.linalg.norm(t, axis=1), r, atol=1e-12)
    assert np.allclose(np.linalg.norm(q, axis=1), 1.0, atol=1e-12)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    approach = R[:, :, 2]
    quarter, above = slice(0, K - 6), slice(K - 6, K)
    assert np.all(t[quarter, 2] > 0) and np.all(t[quarter, 0] >= -1e-12)
    assert np.allclose(approach[quarter], -t[quarter] / r, atol=1e-12)          # facing the CoM
    assert np.allclose(t[above], [0, 0, r], atol=1e-12)
    assert np.allclose(approach[above], [0, 0, -1], atol=1e-12)
    yaw = np.degrees(np.arctan2(R[above, 1, 0], R[above, 0, 0]))
    assert np.allclose(np.diff(np.unwrap(np.radians(yaw))), np.radians(60.0), atol=1e-9)
    # area-uniform lattice: the z coordinates are the midpoints of n equal bands
    n = K - 6
    assert np.allclose(np.sort(t[quarter, 2] / r)[::-1], 1 - (np.arange(n) + 0.5) / n, atol=1e-12)


def test_priors_in_the_stein_direction_closed_form():
    """K = 1, no cost gradient: phi = gamma grad log p = gamma (-(t - CoM)/sigma^2, kappa sign(mu.q)
    projected mu) (plus the self-repulsion, radial in q, which the projection removes)."""
    import oracle
    g = np.random.default_rng(21)
    com = np.array([0.02, -0.01, 0.05])
    mu = np.array([0.3, -0.4, 0.5, 0.7]); mu /= np.linalg.norm(mu)
    th = np.zeros((1, 7)); th[0, :3] = com + g.normal(0, 0.05, 3)
    q = g.normal(size=4); q /= np.linalg.norm(q); th[0, 3:] = -q if q @ mu > 0 else q   # mu.q < 0
    sigma, kappa, gam = 0.07, 3.0, 0.6
    phi = oracle.stein_direction(th, np.zeros((1, 7)), 100, gam, 1.0, prior=(sigma, kappa, mu, com))[0]
    qq = th[0, 3:]
    assert np.allclose(phi[:3], -gam * (th[0, :3] - com) / sigma ** 2, rtol=1e-12, atol=0)
    d = -kappa * mu                                     # sign(mu.q) = -1
    assert np.allclose(phi[3:], gam * (d - (d @ qq) * qq), rtol=1e-12, atol=1e-15)
    # switched off, the priors change nothing
    grad = g.normal(size=(5, 7)); th5 = np.tile(th, (5, 1)); th5[:, :3] += g.normal(0, 0.03, (5, 3))
    a = oracle.stein_direction(th5, grad, 100, gam, 0.01)
    b = oracle.stein_direction(th5, grad, 100, gam, 0.01, prior=(0.0, 0.0, mu, com))
    assert np.array_equal(a, b)


def test_minibatch_ramp_follows_table1():
    """m_k = ceil(M min(k, 2 k_max/3) / (2 k_max/3)), at least one point, ascending unique indices."""
    from paper_2412_08346_gb300 import synth
    M, k_max = 1000, 30
    off, idx = synth.minibatch_ramp(M, k_max, 3)
    sizes = np.diff(off)
    ramp = 2 * k_max / 3
    want = [min(max(int(np.ceil(M * min(k, ramp) / ramp)), 1), M) for k in range(k_max)]
    assert list(sizes) == want and sizes[0] == 1 and sizes[-1] == M
    for k in range(k_max):
        sub = idx[off[k]:off[k + 1]]
        assert np.all(np.diff(sub) > 0) and sub[0] >= 0 and sub[-1] < M


def test_match_cost_with_a_given_com():
    """A mini-batch of R keeps the whole object's CoM: the cost with an explicit CoM equals the
    formula of Eqs. 13-15 written out with brute-force correspondences into the mini-batch."""
    import oracle
    g = np.random.default_rng(31)
    S = g.normal(0, 0.03, (1, 30, 3))
    R = g.normal(0, 0.05, (200, 3))
    sub = R[::3]
    com = R.mean(0)
    grid = np.zeros((4, 4, 4))
    o = oracle.Oracle(S, [(grid, np.array([-1.0, -1, -1]), 0.5)], sub, Cc=R, K=1, com=com)
    th = np.array([0.01, -0.02, 0.03, 0.9, 0.1, -0.2, 0.3]); th[3:] /= np.linalg.norm(th[3:])
    Rm = Rotation.from_quat(th[[4, 5, 6, 3]]).as_matrix()
    sp = S[0] @ Rm.T + th[:3]
    d2 = ((sp[:, None, :] - sub[None]) ** 2).sum(-1)
    nn = d2.argmin(1)
    tcp = S[0].mean(0)
    ref = (d2[np.arange(30), nn].sum() + ((Rm @ tcp + th[:3] - com) ** 2).sum()) / 30
    cost, _ = o.match_terms(0, th, nn.astype(np.int32))
    assert abs(cost - ref) <= 1e-12 * ref


# ------------------------------------------------------------------ convergence (Table I, Section IV-D)
CONV_TOL = 2e-4            # Table I: convergence criterion 0.02 %


def _three_particles(oracle_mod, g):
    orc = _tiny_problem(oracle_mod, g, K=3)
    th = np.stack([np.concatenate([g.uniform(-0.03, 0.03, 3) + [0, 0, 0.2], rand_quat(g)]) for _ in range(3)])
    return orc, th


def test_convergence_threshold_freezes_below_and_not_above(oracle_mod):
    """SGD phase: a particle whose relative cost change |L_k - L_(k-1)| / L_(k-1) is just below the
    criterion stops (its pose is kept exactly), one just above takes the full SGD step; the
    change counts in either direction.  L_k is computed independently by the per-particle cost."""
    g = np.random.default_rng(40)
    orc, th = _three_particles(oracle_mod, g)
    L = np.array([orc.match_cost_grad(0, th[j])[0] for j in range(3)])
    grads = np.stack([orc.match_cost_grad(0, th[j])[1] for j in range(3)])
    for sign in (1.0, -1.0):
        # relative changes 0.9, 1.1 and 0.5 x the criterion (prev above or below L)
        rel = np.array([0.9, 1.1, 0.5]) * CONV_TOL
        prev = L / (1.0 + sign * rel)
        st = orc.new_state(th[None])
        st["prev_cost"][0] = prev
        orc.step(st, orc.schedule(k_max=4, k_stein=1, N=orc.N, conv_tol=CONV_TOL), 2)
        assert st["frozen"][0].tolist() == [1, 0, 1]
        assert np.array_equal(st["theta"][0, 0], th[0]) and np.array_equal(st["theta"][0, 2], th[2])
        new = th[1] - grads[1]
        new[3:] /= np.linalg.norm(new[3:])
        assert np.allclose(st["theta"][0, 1], new, atol=1e-15)
        assert np.array_equal(st["prev_cost"][0], L)       # the next step compares against this cost
    # conv_tol < 0 switches freezing off: every particle steps
    st = orc.new_state(th[None])
    st["prev_cost"][0] = L
    orc.step(st, orc.schedule(k_max=4, k_stein=1, N=orc.N, conv_tol=-1.0), 2)
    assert st["frozen"][0].tolist() == [0, 0, 0]
    assert not np.array_equal(st["theta"][0, 0], th[0])


def test_no_freeze_in_the_svgd_phase_or_without_a_previous_cost(oracle_mod):
    """Nothing freezes while k < k_stein (the SVGD update moves every particle, Eq. 7), nor at the
    first step of a run, where no previous cost exists (prev_cost < 0)."""
    g = np.random.default_rng(41)
    orc, th = _three_particles(oracle_mod, g)
    L = np.array([orc.match_cost_grad(0, th[j])[0] for j in range(3)])
    st = orc.new_state(th[None])
    st["prev_cost"][0] = L                       # zero relative change
    orc.step(st, orc.schedule(k_max=4, k_stein=2, N=orc.N, conv_tol=CONV_TOL), 1)
    assert st["frozen"][0].tolist() == [0, 0, 0]
    assert all(not np.array_equal(st["theta"][0, j], th[j]) for j in range(3))
    st = orc.new_state(th[None])                 # prev_cost = -1
    orc.step(st, orc.schedule(k_max=4, k_stein=0, N=orc.N, conv_tol=1.0), 0)
    assert st["frozen"][0].tolist() == [0, 0, 0]


def test_collision_unfreezes_a_particle(oracle_mod):
    """Section IV-D: a frozen particle whose gripper collides is set back to unconverged and takes the
    collision step (Eq. 18), even with no change in its cost."""
    pts = [[0.001, 0.001, -0.005], [0.0, 0.0, 0.05]]
    orc, S = _palm_problem(oracle_mod, pts)
    th = np.array([0, 0, 0, 1.0, 0, 0, 0])
    lst, _ = orc.collision_points(0, th)
    Lc, gc, _ = orc.collision_cost_grad(0, th, lst)
    st = orc.new_state(th[None, None])
    st["frozen"][0, 0] = 1
    st["prev_cost"][0, 0] = Lc
    orc.step(st, orc.schedule(k_max=2, k_stein=0, N=orc.N, conv_tol=CONV_TOL), 1)
    assert st["ncol"][0, 0] == 1 and st["frozen"][0, 0] == 0
    new = th - gc
    new[3:] /= np.linalg.norm(new[3:])
    assert np.allclose(st["theta"][0, 0], new, atol=1e-15)
    # without the collision the same frozen particle stays where it is
    orc2, _ = _palm_problem(oracle_mod, [[0.0, 0.0, 0.05]])
    L2 = orc2.match_cost_grad(0, th)[0]
    st = orc2.new_state(th[None, None])
    st["frozen"][0, 0] = 1
    st["prev_cost"][0, 0] = L2
    orc2.step(st, orc2.schedule(k_max=2, k_stein=0, N=orc2.N, conv_tol=CONV_TOL), 1)
    assert st["frozen"][0, 0] == 1 and np.array_equal(st["theta"][0, 0], th)


def test_freezing_run_matches_the_free_run_up_to_the_criterion(oracle_mod):
    """SGD-ICP on the known-transform problem, once with freezing and once without: the two runs are
    identical up to the first iteration k* >= 1 at which the free run's cost sequence meets the
    criterion; from k* on the frozen run's pose and cost no longer change."""
    g = np.random.default_rng(12)
    N = 20
    S = g.uniform(-0.5, 0.5, (N, 3))
    R_true = Rotation.from_rotvec([0.3, -0.2, 0.1]).as_matrix()
    t_true = np.array([0.1, 0.2, -0.1])
    obj = S @ R_true.T + t_true + g.normal(0, 1e-3, (N, 3))     # noisy: the cost settles above 0
    grid = -np.ones((4, 4, 4))
    orc = oracle_mod.Oracle(S[None], [(grid, np.full(3, -5.0), 10.0 / 3)], obj, K=1, w_com=0.0)
    xyzw = Rotation.from_matrix(R_true).as_quat()
    q0 = np.array([xyzw[3], xyzw[0], xyzw[1], xyzw[2]]) + np.array([0.0, 0.02, -0.01, 0.015])
    th0 = np.concatenate([t_true + [0.03, -0.02, 0.01], q0 / np.linalg.norm(q0)])
    n_it = 60
    free, frz = orc.new_state(th0[None, None]), orc.new_state(th0[None, None])
    sf, sz = (orc.schedule(k_max=n_it, k_stein=0, N=N, conv_tol=c) for c in (-1.0, CONV_TOL))
    costs, thetas_free, thetas_frz, frozen = [], [], [], []
    for k in range(n_it):
        orc.step(free, sf, k)
        orc.step(frz, sz, k)
        costs.append(free["cost"][0, 0])
        thetas_free.append(free["theta"][0, 0].copy())
        thetas_frz.append(frz["theta"][0, 0].copy())
        frozen.append(int(frz["frozen"][0, 0]))
    kstar = next(k for k in range(1, n_it) if abs(costs[k] - costs[k - 1]) <= CONV_TOL * costs[k - 1])
    assert 1 <= kstar < n_it - 5
    assert frozen[:kstar] == [0] * kstar and frozen[kstar:] == [1] * (n_it - kstar)
    for k in range(kstar):
        assert np.array_equal(thetas_frz[k], thetas_free[k])
    for k in range(kstar, n_it):
        assert np.array_equal(thetas_frz[k], thetas_free[kstar - 1])


def test_convergence_criterion_includes_equality(oracle_mod):
    """Reading of Table I's 0.02 %: a relative change equal to the criterion counts as converged
    (|L_k - L_(k-1)| <= tol L_(k-1)).  With tol = 0 only an unchanged cost meets it: equality
    freezes, the smallest change in either direction does not."""
    g = np.random.default_rng(42)
    orc, th = _three_particles(oracle_mod, g)
    L = np.array([orc.match_cost_grad(0, th[j])[0] for j in range(3)])
    st = orc.new_state(th[None])
    st["prev_cost"][0] = [L[0], np.nextafter(L[1], np.inf), np.nextafter(L[2], -np.inf)]
    orc.step(st, orc.schedule(k_max=4, k_stein=1, N=orc.N, conv_tol=0.0), 2)
    assert st["frozen"][0].tolist() == [1, 0, 0]


def test_decision_margin_brute_force(oracle_mod):
    """The decision margin the free-running tests use to tell near-tie particles apart: the smallest
    of the nearest-vs-runner-up distance gaps of every gripper point (Eq. 1), |SDF| of every
    collision point inside the grid (Eq. 12) and the gaps of the colliding points' reverse matches
    (Eq. 18), against numpy on a palm problem with a colliding point and a planted exact tie."""
    pts = np.array([[0.001, 0.001, -0.005], [0.0, 0.0, 0.05], [0.03, -0.02, 0.01]])
    orc, S = _palm_problem(oracle_mod, pts)
    for th in (np.array([0, 0, 0, 1.0, 0, 0, 0]), np.array([0.002, -0.001, 0.003, 0.99, 0.1, 0.0, 0.05])):
        th = th.copy()
        th[3:] /= np.linalg.norm(th[3:])
        R = Rotation.from_quat([th[4], th[5], th[6], th[3]]).as_matrix()
        Sp = S.astype(np.float64) @ R.T + th[:3]
        d = np.sqrt(((Sp[:, None, :] - orc.R[None]) ** 2).sum(-1))
        ds = np.sort(d, axis=1)
        m = (ds[:, 1] - ds[:, 0]).min()
        lst, vals = orc.collision_points(0, th)
        xg = (pts - th[:3]) @ R                        # collision points in the gripper frame
        sdf, origin, voxel = synth.sdf_grid(0.0, 41)
        n = np.array(sdf.shape[::-1])
        inside = np.all((xg - origin) / voxel >= 0, 1) & np.all((xg - origin) / voxel <= n - 1, 1)
        m = min(m, np.abs(vals[inside]).min())
        for c in lst:
            dc = np.sort(np.sqrt(((Sp - pts[c]) ** 2).sum(-1)))
            m = min(m, dc[1] - dc[0])
        assert orc.decision_margin(0, th) == pytest.approx(m, rel=1e-12, abs=1e-15)
        st = orc.new_state(th[None, None], margin=True)
        orc.evaluate(st)
        assert st["margin"][0, 0] == orc.decision_margin(0, th)
    # a planted duplicate object point is an exact tie: margin 0
    orc2, _ = _palm_problem(oracle_mod, np.concatenate([pts, pts[2:3]]))
    assert orc2.decision_margin(0, np.array([0, 0, 0, 1.0, 0, 0, 0])) == 0.0
