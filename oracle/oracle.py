"""ctypes wrapper around the FP64 oracle (``asicp_oracle.c``).  Test infrastructure only."""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "asicp_oracle.c")
_HDR = os.path.join(_HERE, "asicp_oracle.h")
_LIB = os.path.join(_HERE, "_build", "libasicp_oracle.so")
_lock = threading.Lock()
_lib = None

_dp = C.POINTER(C.c_double)
_ip = C.POINTER(C.c_int)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C, OpenMP over particles)."""
    with _lock:
        newest = max(os.path.getmtime(_SRC), os.path.getmtime(_HDR))
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < newest:
            os.makedirs(os.path.dirname(_LIB), exist_ok=True)
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-ffp-contract=off",
                                   "-fno-fast-math", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


class _Problem(C.Structure):
    _fields_ = [("P", C.c_int), ("K", C.c_int), ("N", C.c_int), ("M", C.c_int), ("Mc", C.c_int),
                ("S", _dp), ("R", _dp), ("C", _dp), ("sdf", _dp), ("sdf_off", C.POINTER(C.c_longlong)),
                ("sdf_dims", _ip), ("sdf_origin", _dp), ("sdf_voxel", _dp), ("w_com", C.c_double),
                ("com", _dp)]


class _Schedule(C.Structure):
    _fields_ = [("k_max", C.c_int), ("k_stein", C.c_int), ("schedule", C.c_int),
                ("C_cycles", C.c_double), ("p_exp", C.c_double), ("g0", C.c_double), ("g1", C.c_double),
                ("eta_sgd", C.c_double), ("eta_svgd", C.c_double), ("bandwidth_mode", C.c_int),
                ("h_fixed", C.c_double), ("conv_tol", C.c_double), ("prior_t_sigma", C.c_double),
                ("prior_q_kappa", C.c_double), ("prior_q_mean", C.c_double * 4)]


class _State(C.Structure):
    _fields_ = [("theta", _dp), ("cost", _dp), ("grad", _dp), ("phi", _dp), ("ncol", _ip),
                ("frozen", _ip), ("prev_cost", _dp), ("h", _dp), ("nn_idx", _ip), ("col_list", _ip),
                ("col_nn", _ip), ("sdf_val", _dp), ("margin", _dp)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        lib.orc_rotation.argtypes = [_dp, _dp]
        lib.orc_rot_jacobian.argtypes = [_dp, _dp, _dp]
        lib.orc_nn.argtypes = [_dp, C.c_int, _dp, C.c_int, _ip, _dp]
        lib.orc_trilinear.argtypes = [_dp, _ip, _dp, C.c_double, _dp, _ip]
        lib.orc_trilinear.restype = C.c_double
        lib.orc_match_cost_grad.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _dp, _dp, _ip]
        lib.orc_collision_points.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _ip, _dp]
        lib.orc_collision_points.restype = C.c_int
        lib.orc_collision_cost_grad.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _ip, C.c_int, _dp, _dp, _ip]
        lib.orc_match_terms.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _ip, _dp, _dp]
        lib.orc_collision_terms.argtypes = [C.POINTER(_Problem), C.c_int, _dp, _ip, _ip, C.c_int, _dp, _dp]
        lib.orc_gamma.argtypes = [C.POINTER(_Schedule), C.c_int]
        lib.orc_gamma.restype = C.c_double
        lib.orc_bandwidth.argtypes = [_dp, C.c_int, C.POINTER(_Schedule)]
        lib.orc_bandwidth.restype = C.c_double
        lib.orc_stein_direction.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_double, C.c_double, _dp]
        lib.orc_stein_direction_prior.argtypes = [_dp, _dp, C.c_int, C.c_int, C.c_double, C.c_double, _dp, _dp]
        lib.orc_fibonacci_init.argtypes = [C.c_int, _dp, C.c_double, _dp]
        lib.orc_quarter_init.argtypes = [C.c_int, _dp, C.c_double, _dp]
        lib.orc_centroid.argtypes = [_dp, C.c_int, _dp]
        lib.orc_step.argtypes = [C.POINTER(_Problem), C.POINTER(_Schedule), C.POINTER(_State), C.c_int, C.c_int]
        lib.orc_evaluate.argtypes = [C.POINTER(_Problem), C.POINTER(_State), C.c_int]
        lib.orc_select.argtypes = [_dp, _ip, C.c_int, C.c_int, _ip]
        lib.orc_decision_margin.argtypes = [C.POINTER(_Problem), C.c_int, _dp]
        lib.orc_decision_margin.restype = C.c_double
        _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(_dp)


def _i(a):
    a = np.ascontiguousarray(a, dtype=np.int32)
    return a, a.ctypes.data_as(_ip)


# ---------------------------------------------------------------- primitives
def rotation(q):
    q, qp = _d(q)
    out = np.zeros(9)
    _load().orc_rotation(qp, out.ctypes.data_as(_dp))
    return out.reshape(3, 3)


def rot_jacobian(q, s):
    q, qp = _d(q)
    s, sp = _d(s)
    out = np.zeros(12)
    _load().orc_rot_jacobian(qp, sp, out.ctypes.data_as(_dp))
    return out.reshape(3, 4)


def nn(queries, refs):
    q, qp = _d(np.asarray(queries).reshape(-1, 3))
    r, rp = _d(np.asarray(refs).reshape(-1, 3))
    idx = np.zeros(len(q), np.int32)
    d2 = np.zeros(len(q))
    _load().orc_nn(qp, len(q), rp, len(r), idx.ctypes.data_as(_ip), d2.ctypes.data_as(_dp))
    return idx, d2


def centroid(X):
    X, xp = _d(np.asarray(X).reshape(-1, 3))
    out = np.zeros(3)
    _load().orc_centroid(xp, len(X), out.ctypes.data_as(_dp))
    return out


def trilinear(grid_zyx, origin, voxel, x):
    g, gp = _d(grid_zyx)
    dims = np.array([grid_zyx.shape[2], grid_zyx.shape[1], grid_zyx.shape[0]], np.int32)
    o, op = _d(origin)
    x, xp = _d(x)
    inside = C.c_int(0)
    v = _load().orc_trilinear(gp, dims.ctypes.data_as(_ip), op, float(voxel), xp, C.byref(inside))
    return v, bool(inside.value)


def gamma(k, k_max, schedule=0, C_cycles=5.0, p_exp=2.0, g0=0.1, g1=1.0):
    sc = _Schedule(k_max, 0, schedule, C_cycles, p_exp, g0, g1, 1.0, 1.0, 0, 1.0, -1.0)
    return _load().orc_gamma(C.byref(sc), int(k))


def bandwidth(theta, bandwidth_mode=0, h_fixed=1.0):
    th, tp = _d(np.asarray(theta).reshape(-1, 7))
    sc = _Schedule(1, 0, 0, 5.0, 2.0, 0.1, 1.0, 1.0, 1.0, bandwidth_mode, h_fixed, -1.0)
    return _load().orc_bandwidth(tp, len(th), C.byref(sc))


def stein_direction(theta, grad, N, gamma_, h, prior=None):
    """prior: None or (sigma_t, kappa_q, mean_q (4), CoM (3))."""
    th, tp = _d(np.asarray(theta).reshape(-1, 7))
    g, gp = _d(np.asarray(grad).reshape(-1, 7))
    phi = np.zeros_like(th)
    if prior is None:
        pp = None
    else:
        pr, pp = _d(np.concatenate([[prior[0], prior[1]], prior[2], prior[3]]).astype(np.float64))
    _load().orc_stein_direction_prior(tp, gp, len(th), int(N), float(gamma_), float(h), pp,
                                      phi.ctypes.data_as(_dp))
    return phi


def fibonacci_init(K, com, radius):
    c, cp = _d(com)
    out = np.zeros((K, 7))
    _load().orc_fibonacci_init(int(K), cp, float(radius), out.ctypes.data_as(_dp))
    return out


def quarter_init(K, com, radius):
    """Quarter-sphere Fibonacci initialisation plus six poses above the object (see the C source)."""
    c, cp = _d(com)
    out = np.zeros((K, 7))
    _load().orc_quarter_init(int(K), cp, float(radius), out.ctypes.data_as(_dp))
    return out


def select(cost, ncol, topk):
    c, cp = _d(cost)
    n, np_ = _i(ncol)
    order = np.full(topk, -1, np.int32)
    _load().orc_select(cp, np_, len(c), int(topk), order.ctypes.data_as(_ip))
    return order


# ---------------------------------------------------------------- problem
class Oracle:
    """Holds one problem (preshape clouds + SDFs, object cloud) in float64.

    ``S`` is (P, N, 3); ``sdfs`` a list of (grid[z, y, x], origin, voxel);
    ``R`` is (M, 3); ``Cc`` the collision cloud (defaults to ``R``).
    """

    def __init__(self, S, sdfs, R, Cc=None, K=1, w_com=1.0, com=None):
        self.S = np.ascontiguousarray(np.asarray(S, dtype=np.float64).reshape(len(S), -1, 3))
        self.P, self.N = self.S.shape[0], self.S.shape[1]
        self.R = np.ascontiguousarray(np.asarray(R, dtype=np.float64).reshape(-1, 3))
        self.Cc = self.R if Cc is None else np.ascontiguousarray(np.asarray(Cc, dtype=np.float64).reshape(-1, 3))
        self.K = int(K)
        grids, offs, dims, orgs, vox = [], [], [], [], []
        off = 0
        for g, o, v in sdfs:
            g = np.asarray(g, dtype=np.float64)
            grids.append(g.ravel())
            offs.append(off)
            off += g.size
            dims.append([g.shape[2], g.shape[1], g.shape[0]])
            orgs.append(np.asarray(o, dtype=np.float64))
            vox.append(float(v))
        self.sdf = np.ascontiguousarray(np.concatenate(grids))
        self.sdf_off = np.ascontiguousarray(np.array(offs, np.int64))
        self.sdf_dims = np.ascontiguousarray(np.array(dims, np.int32))
        self.sdf_origin = np.ascontiguousarray(np.array(orgs, np.float64))
        self.sdf_voxel = np.ascontiguousarray(np.array(vox, np.float64))
        self.w_com = float(w_com)
        self._com = None if com is None else np.ascontiguousarray(np.asarray(com, dtype=np.float64).reshape(3))
        self._pb = _Problem(self.P, self.K, self.N, len(self.R), len(self.Cc),
                            self.S.ctypes.data_as(_dp), self.R.ctypes.data_as(_dp), self.Cc.ctypes.data_as(_dp),
                            self.sdf.ctypes.data_as(_dp), self.sdf_off.ctypes.data_as(C.POINTER(C.c_longlong)),
                            self.sdf_dims.ctypes.data_as(_ip), self.sdf_origin.ctypes.data_as(_dp),
                            self.sdf_voxel.ctypes.data_as(_dp), self.w_com,
                            None if com is None else self._com.ctypes.data_as(_dp))

    # ---- per particle
    def match_cost_grad(self, p, theta):
        th, tp = _d(theta)
        cost = C.c_double(0)
        g = np.zeros(7)
        idx = np.zeros(self.N, np.int32)
        _load().orc_match_cost_grad(C.byref(self._pb), int(p), tp, C.byref(cost), g.ctypes.data_as(_dp),
                                    idx.ctypes.data_as(_ip))
        return cost.value, g, idx

    def match_terms(self, p, theta, nn_idx):
        """Cost and gradient for given pairs (gripper point i <-> object point nn_idx[i])."""
        th, tp = _d(theta)
        idx, ip = _i(nn_idx)
        cost = C.c_double(0)
        g = np.zeros(7)
        _load().orc_match_terms(C.byref(self._pb), int(p), tp, ip, C.byref(cost), g.ctypes.data_as(_dp))
        return cost.value, g

    def collision_terms(self, p, theta, lst, nn_):
        """Collision cost and gradient for given pairs (C[lst[l]] <-> gripper point nn_[l])."""
        th, tp = _d(theta)
        lst, lp = _i(lst)
        nn_, np_ = _i(nn_)
        cost = C.c_double(0)
        g = np.zeros(7)
        _load().orc_collision_terms(C.byref(self._pb), int(p), tp, lp, np_, len(lst), C.byref(cost),
                                    g.ctypes.data_as(_dp))
        return cost.value, g

    def collision_points(self, p, theta):
        th, tp = _d(theta)
        lst = np.zeros(max(1, len(self.Cc)), np.int32)
        vals = np.zeros(len(self.Cc))
        n = _load().orc_collision_points(C.byref(self._pb), int(p), tp, lst.ctypes.data_as(_ip),
                                         vals.ctypes.data_as(_dp))
        return lst[:n].copy(), vals

    def collision_cost_grad(self, p, theta, lst):
        th, tp = _d(theta)
        lst, lp = _i(lst)
        cost = C.c_double(0)
        g = np.zeros(7)
        nn_ = np.zeros(max(1, len(lst)), np.int32)
        _load().orc_collision_cost_grad(C.byref(self._pb), int(p), tp, lp, len(lst), C.byref(cost),
                                        g.ctypes.data_as(_dp), nn_.ctypes.data_as(_ip))
        return cost.value, g, nn_[:len(lst)].copy()

    # ---- whole iterations
    def decision_margin(self, p, theta):
        """Smallest gap (metres) by which the step's discrete decisions at theta could change."""
        th, tp = _d(theta)
        return _load().orc_decision_margin(C.byref(self._pb), int(p), tp)

    def new_state(self, theta, debug=False, margin=False):
        P, K = self.P, self.K
        st = {
            "theta": np.ascontiguousarray(np.asarray(theta, dtype=np.float64).reshape(P, K, 7).copy()),
            "cost": np.zeros((P, K)), "grad": np.zeros((P, K, 7)), "phi": np.zeros((P, K, 7)),
            "ncol": np.zeros((P, K), np.int32), "frozen": np.zeros((P, K), np.int32),
            "prev_cost": np.full((P, K), -1.0), "h": np.zeros(P),
        }
        if debug:
            st["nn_idx"] = np.zeros((P, K, self.N), np.int32)
            st["col_list"] = np.zeros((P, K, len(self.Cc)), np.int32)
            st["col_nn"] = np.zeros((P, K, len(self.Cc)), np.int32)
            st["sdf_val"] = np.zeros((P, K, len(self.Cc)))
        if margin:
            st["margin"] = np.zeros((P, K))
        return st

    def _cstate(self, st):
        def dp(k):
            return st[k].ctypes.data_as(_dp) if k in st else None

        def ip(k):
            return st[k].ctypes.data_as(_ip) if k in st else None
        return _State(dp("theta"), dp("cost"), dp("grad"), dp("phi"), ip("ncol"), ip("frozen"),
                      dp("prev_cost"), dp("h"), ip("nn_idx"), ip("col_list"), ip("col_nn"), dp("sdf_val"),
                      dp("margin"))

    @staticmethod
    def schedule(k_max, k_stein, schedule=0, C_cycles=5.0, p_exp=2.0, g0=0.1, g1=1.0, eta_sgd=1.0,
                 eta_svgd=None, N=1, bandwidth_mode=0, h_fixed=1.0, conv_tol=-1.0, prior_t_sigma=0.0,
                 prior_q_kappa=0.0, prior_q_mean=(1.0, 0.0, 0.0, 0.0)):
        if eta_svgd is None:
            eta_svgd = 1.0 / N
        return _Schedule(int(k_max), int(k_stein), int(schedule), C_cycles, p_exp, g0, g1, eta_sgd, eta_svgd,
                         int(bandwidth_mode), h_fixed, conv_tol, prior_t_sigma, prior_q_kappa,
                         (C.c_double * 4)(*prior_q_mean))

    def step(self, st, sched, k, nthreads=1):
        cs = self._cstate(st)
        _load().orc_step(C.byref(self._pb), C.byref(sched), C.byref(cs), int(k), int(nthreads))
        return st

    def evaluate(self, st, nthreads=1):
        cs = self._cstate(st)
        _load().orc_evaluate(C.byref(self._pb), C.byref(cs), int(nthreads))
        return st

    def run(self, theta0, sched, nthreads=1, topk=8):
        st = self.new_state(theta0)
        for k in range(sched.k_max):
            self.step(st, sched, k, nthreads)
        self.evaluate(st, nthreads)
        order = select(st["cost"].ravel(), st["ncol"].ravel(), topk)
        return st, order
