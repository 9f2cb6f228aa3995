"""Thin ctypes binding of libasicp (include/asicp.h): argument marshalling only.

Every function has the name of the C entry point it calls.  Arrays may be
torch tensors (CPU or CUDA; contiguous float32 / int32 / float64 as the C
declaration says) or numpy arrays; their addresses are passed straight
through, so the library sees host or device memory exactly as the caller
holds it.  There is no fallback: if the shared library is missing, importing
the binding raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

ASICP_OK = 0
ASICP_ERR_INVALID_ARG = 1
ASICP_ERR_STATE = 2
ASICP_ERR_CUDA = 3
ASICP_ERR_OOM = 4
ASICP_ERR_TIMEOUT = 5
STATUS_NAMES = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "CUDA", 4: "OOM", 5: "TIMEOUT"}

EXPORTED = ("asicp_config_default", "asicp_create", "asicp_destroy", "asicp_set_object",
            "asicp_set_gripper_sdf", "asicp_set_state", "asicp_step", "asicp_run", "asicp_best_grasps",
            "asicp_get_state", "asicp_kernel_times", "asicp_last_error", "asicp_match_noalloc",
            "asicp_set_object_at", "asicp_set_particle_counts", "asicp_best_grasps_at", "asicp_autotune",
            "asicp_set_minibatch", "asicp_set_convergence", "asicp_test_expire_waits")


class AsicpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class asicp_config(C.Structure):
    _fields_ = [("P", C.c_int), ("K", C.c_int), ("k_max", C.c_int), ("k_stein", C.c_int),
                ("schedule", C.c_int), ("C_cycles", C.c_float), ("p_exp", C.c_float), ("g0", C.c_float),
                ("g1", C.c_float), ("eta_sgd", C.c_float), ("eta_svgd", C.c_float), ("w_com", C.c_float),
                ("bandwidth_mode", C.c_int), ("h_fixed", C.c_float), ("conv_tol", C.c_float),
                ("init_radius", C.c_float), ("debug", C.c_int), ("profile", C.c_int),
                ("cuda_stream", C.c_void_p), ("n_objects", C.c_int), ("autotune", C.c_int), ("fwd_shape", C.c_int), ("init_mode", C.c_int),
                ("prior_t_sigma", C.c_float), ("prior_q_kappa", C.c_float), ("prior_q_mean", C.c_float * 4)]


class asicp_state_view(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("cost", C.c_void_p), ("grad", C.c_void_p), ("phi", C.c_void_p),
                ("ncol", C.c_void_p), ("frozen", C.c_void_p), ("h", C.c_void_p), ("nn_idx", C.c_void_p),
                ("nn_d2", C.c_void_p), ("s_prime", C.c_void_p), ("col_list", C.c_void_p),
                ("col_nn", C.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libasicp.so (building it first when asked and the sources are newer)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libasicp.so not found at {_build.LIB}: run paper_2412_08346_gb300.build.build()")
    lib = C.CDLL(_build.LIB)
    vp, ip = C.c_void_p, C.c_int
    lib.asicp_config_default.argtypes = [C.POINTER(asicp_config)]
    lib.asicp_config_default.restype = None
    lib.asicp_create.argtypes = [C.POINTER(asicp_config), C.POINTER(vp)]
    lib.asicp_destroy.argtypes = [vp]
    lib.asicp_set_object.argtypes = [vp, vp, ip, vp, ip]
    lib.asicp_set_gripper_sdf.argtypes = [vp, ip, vp, ip, vp, ip, ip, ip, vp, C.c_float]
    lib.asicp_set_state.argtypes = [vp, vp, ip]
    lib.asicp_set_convergence.argtypes = [vp, vp, vp]
    lib.asicp_test_expire_waits.argtypes = [vp, ip]
    lib.asicp_step.argtypes = [vp, ip]
    lib.asicp_run.argtypes = [vp, vp]
    lib.asicp_best_grasps.argtypes = [vp, ip, vp, vp, vp, C.POINTER(C.c_int)]
    lib.asicp_get_state.argtypes = [vp, C.POINTER(asicp_state_view)]
    lib.asicp_kernel_times.argtypes = [vp, C.POINTER(C.c_double), C.POINTER(C.c_longlong), ip]
    lib.asicp_match_noalloc.argtypes = [vp, ip, ip, vp, ip, vp, ip, vp, vp]
    lib.asicp_set_object_at.argtypes = [vp, ip, vp, ip, vp, ip]
    lib.asicp_autotune.argtypes = [vp, C.POINTER(C.c_int), C.POINTER(C.c_float)]
    lib.asicp_set_minibatch.argtypes = [vp, vp, vp, C.c_int]
    lib.asicp_set_particle_counts.argtypes = [vp, vp, ip]
    lib.asicp_best_grasps_at.argtypes = [vp, ip, ip, vp, vp, vp, C.POINTER(C.c_int)]
    lib.asicp_last_error.argtypes = [vp]
    lib.asicp_last_error.restype = C.c_char_p
    for name in EXPORTED:
        if name not in ("asicp_config_default", "asicp_last_error"):
            getattr(lib, name).restype = C.c_int
    _lib = lib
    return lib


def _ptr(a):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("arrays passed to libasicp must be contiguous")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libasicp must be contiguous")
        return a.ctypes.data
    raise TypeError(f"unsupported array type {type(a)}")


def _check(ctx, status):
    if status != ASICP_OK:
        msg = _lib.asicp_last_error(ctx).decode() if ctx else "NULL context"
        raise AsicpError(status, msg)


# ------------------------------------------------------------------ entry points
def asicp_config_default(**overrides) -> asicp_config:
    cfg = asicp_config()
    load().asicp_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def asicp_create(cfg: asicp_config):
    out = C.c_void_p()
    st = load().asicp_create(C.byref(cfg), C.byref(out))
    if st != ASICP_OK:
        raise AsicpError(st, "asicp_create rejected the configuration")
    return out.value


def asicp_destroy(ctx) -> None:
    load().asicp_destroy(ctx)


def asicp_set_object(ctx, R_xyz, C_xyz=None) -> None:
    M = int(R_xyz.shape[0])
    Mc = int(C_xyz.shape[0]) if C_xyz is not None else 0
    _check(ctx, load().asicp_set_object(ctx, _ptr(R_xyz), M, _ptr(C_xyz), Mc))


def asicp_set_object_at(ctx, obj: int, R_xyz, C_xyz=None) -> None:
    M = int(R_xyz.shape[0])
    Mc = int(C_xyz.shape[0]) if C_xyz is not None else 0
    _check(ctx, load().asicp_set_object_at(ctx, int(obj), _ptr(R_xyz), M, _ptr(C_xyz), Mc))


def asicp_set_particle_counts(ctx, K) -> None:
    """``K`` int32 array of n_objects * P particle counts (object-major)."""
    K = np.ascontiguousarray(np.asarray(K, dtype=np.int32))
    _check(ctx, load().asicp_set_particle_counts(ctx, _ptr(K), int(K.size)))


def asicp_set_minibatch(ctx, offsets, indices) -> None:
    """Per-iteration mini-batches of the object cloud: int32 offsets [iters + 1] and ascending
    indices (None switches them off)."""
    if offsets is None:
        _check(ctx, load().asicp_set_minibatch(ctx, None, None, 0))
        return
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32))
    idx = np.ascontiguousarray(np.asarray(indices, dtype=np.int32))
    _check(ctx, load().asicp_set_minibatch(ctx, _ptr(off), _ptr(idx), int(off.size) - 1))


def asicp_set_gripper_sdf(ctx, preshape, S_xyz, sdf_zyx, origin, voxel) -> None:
    """``sdf_zyx`` has shape (nz, ny, nx) (x fastest in memory)."""
    nz, ny, nx = (int(d) for d in sdf_zyx.shape)
    org = np.ascontiguousarray(np.asarray(origin, dtype=np.float32).reshape(3))
    _check(ctx, load().asicp_set_gripper_sdf(ctx, int(preshape), _ptr(S_xyz), int(S_xyz.shape[0]), _ptr(sdf_zyx),
                                             nx, ny, nz, _ptr(org), float(voxel)))


def asicp_set_state(ctx, theta, k: int) -> None:
    _check(ctx, load().asicp_set_state(ctx, _ptr(theta), int(k)))


def asicp_set_convergence(ctx, prev_cost=None, frozen=None) -> None:
    _check(ctx, load().asicp_set_convergence(ctx, _ptr(prev_cost), _ptr(frozen)))


def asicp_test_expire_waits(ctx, on: bool) -> None:
    _check(ctx, load().asicp_test_expire_waits(ctx, int(bool(on))))


def asicp_step(ctx, k: int) -> None:
    _check(ctx, load().asicp_step(ctx, int(k)))


def asicp_run(ctx, theta0=None) -> None:
    _check(ctx, load().asicp_run(ctx, _ptr(theta0)))


def asicp_best_grasps(ctx, topk: int, theta=None, cost=None, preshape=None) -> int:
    n = C.c_int(0)
    _check(ctx, load().asicp_best_grasps(ctx, int(topk), _ptr(theta), _ptr(cost), _ptr(preshape), C.byref(n)))
    return n.value


def asicp_best_grasps_at(ctx, obj: int, topk: int, theta=None, cost=None, preshape=None) -> int:
    n = C.c_int(0)
    _check(ctx, load().asicp_best_grasps_at(ctx, int(obj), int(topk), _ptr(theta), _ptr(cost), _ptr(preshape),
                                            C.byref(n)))
    return n.value


def asicp_get_state(ctx, **arrays) -> None:
    """Fill the given arrays (keyword names of asicp_state_view)."""
    view = asicp_state_view(**{k: _ptr(v) for k, v in arrays.items()})
    _check(ctx, load().asicp_get_state(ctx, C.byref(view)))


KERNEL_KINDS = ("match", "collide", "collide_nn", "finalize", "stein", "exact")


def asicp_kernel_times(ctx, reset: bool = False):
    ms = (C.c_double * len(KERNEL_KINDS))()
    n = (C.c_longlong * len(KERNEL_KINDS))()
    _check(ctx, load().asicp_kernel_times(ctx, ms, n, int(reset)))
    return list(ms), list(n)


def asicp_match_noalloc(theta, S_xyz, R_xyz, nn_idx, P: int, K: int, stream=None) -> None:
    """Nearest-neighbour indices without any device allocation (see include/asicp.h).

    ``theta`` (P*K, 7), ``S_xyz`` (P*N, 3), ``R_xyz`` (M, 3); ``nn_idx`` a CUDA int32 tensor of P*K*N."""
    N = int(S_xyz.shape[0]) // int(P)
    st = load().asicp_match_noalloc(_ptr(theta), int(P), int(K), _ptr(S_xyz), N, _ptr(R_xyz),
                                    int(R_xyz.shape[0]), _ptr(nn_idx), stream)
    if st != ASICP_OK:
        raise AsicpError(st, "asicp_match_noalloc failed")


FWD_VARIANTS = ("qpt8-chunk64-t128-tile2048", "qpt8-chunk32-t128-tile2048", "qpt4-chunk64-t256-tile2048",
                "qpt4-chunk32-t256-tile2048", "qpt4-chunk64-t128-tile1024", "qpt8-chunk64-t128-tile1024",
                "qpt6-chunk64-t128-tile1024", "tc-f16x3-m128-n256")
FWD_SHAPES = len(FWD_VARIANTS)          # ASICP_FWD_SHAPES


def asicp_autotune(ctx):
    """Pick the fastest forward-matching kernel shape; returns (index, [ms per shape])."""
    chosen = C.c_int(0)
    ms = (C.c_float * FWD_SHAPES)()
    _check(ctx, load().asicp_autotune(ctx, C.byref(chosen), ms))
    return chosen.value, list(ms)


def asicp_last_error(ctx) -> str:
    return load().asicp_last_error(ctx).decode()
