"""ctypes binding of the learned initial-pose proposal (include/asicp_proposal.h).

Argument marshalling only: the network's forward and backward passes, its loss,
the Adam step and the sampling all run in the library's CUDA kernels.  Arrays
may be torch tensors (host or CUDA) or numpy arrays, float32, C-contiguous.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import asicp

PROP_EXPORTED = ("asicp_prop_num_params", "asicp_prop_create", "asicp_prop_destroy", "asicp_prop_set_params",
                 "asicp_prop_get_params", "asicp_prop_forward", "asicp_prop_loss_grad", "asicp_prop_adam_step",
                 "asicp_prop_sample")
COMPONENTS = 16
RAW = 10
MAX_TARGETS = 128

_ready = False


def _lib():
    global _ready
    lib = asicp.load()
    if not _ready:
        vp, fp = C.c_void_p, C.c_void_p
        lib.asicp_prop_num_params.argtypes = [C.c_int]
        lib.asicp_prop_num_params.restype = C.c_size_t
        lib.asicp_prop_create.argtypes = [C.c_int, C.c_int, C.c_int, vp, C.POINTER(C.c_void_p)]
        lib.asicp_prop_destroy.argtypes = [vp]
        lib.asicp_prop_set_params.argtypes = [vp, fp]
        lib.asicp_prop_get_params.argtypes = [vp, fp]
        lib.asicp_prop_forward.argtypes = [vp, fp, C.c_int, fp, fp]
        lib.asicp_prop_loss_grad.argtypes = [vp, fp, fp, C.c_int, C.c_int, C.POINTER(C.c_float), fp]
        lib.asicp_prop_adam_step.argtypes = [vp, C.c_float]
        lib.asicp_prop_sample.argtypes = [vp, fp, fp, C.c_int, C.c_int, fp, fp]
        for n in PROP_EXPORTED[1:]:
            getattr(lib, n).restype = C.c_int
        _ready = True
    return lib


def num_params(P: int) -> int:
    return int(_lib().asicp_prop_num_params(P))


def _ok(status, what):
    if status != asicp.ASICP_OK:
        raise asicp.AsicpError(status, what)


class Proposal:
    """The proposal network for P preshapes and clouds of n_points points."""

    def __init__(self, P: int, n_points: int, max_batch: int, stream=None):
        self.h = None
        self.P, self.n_points, self.max_batch = P, n_points, max_batch
        h = C.c_void_p()
        _ok(_lib().asicp_prop_create(P, n_points, max_batch, stream, C.byref(h)), "asicp_prop_create")
        self.h = h
        self.n_params = num_params(P)

    def close(self):
        if getattr(self, "h", None):
            _lib().asicp_prop_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_params(self, params):
        _ok(_lib().asicp_prop_set_params(self.h, asicp._ptr(params)), "asicp_prop_set_params")

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.n_params, np.float32)
        _ok(_lib().asicp_prop_get_params(self.h, asicp._ptr(out)), "asicp_prop_get_params")
        return out

    def forward(self, clouds, B: int, out=None, centroids=None):
        """Raw mixture outputs [B, P, 16, 10] and centroids [B, 3] (numpy unless buffers are given)."""
        if out is None:
            out = np.zeros((B, self.P, COMPONENTS, RAW), np.float32)
        if centroids is None:
            centroids = np.zeros((B, 3), np.float32)
        _ok(_lib().asicp_prop_forward(self.h, asicp._ptr(clouds), B, asicp._ptr(out), asicp._ptr(centroids)),
            "asicp_prop_forward")
        return out, centroids

    def loss_grad(self, clouds, targets, B: int, T: int, want_grad: bool = False):
        loss = C.c_float(0.0)
        grad = np.zeros(self.n_params, np.float32) if want_grad else None
        _ok(_lib().asicp_prop_loss_grad(self.h, asicp._ptr(clouds), asicp._ptr(targets), B, T, C.byref(loss),
                                        asicp._ptr(grad)), "asicp_prop_loss_grad")
        return float(loss.value), grad

    def adam_step(self, lr: float):
        _ok(_lib().asicp_prop_adam_step(self.h, float(lr)), "asicp_prop_adam_step")

    def sample(self, out, centroids, B: int, K: int, draws, theta=None):
        """Initial poses [B, P, K, 7] from the mixtures; draws [B, P, K, 8] = (u, 7 normals)."""
        if theta is None:
            theta = np.zeros((B, self.P, K, 7), np.float32)
        _ok(_lib().asicp_prop_sample(self.h, asicp._ptr(out), asicp._ptr(centroids), B, K, asicp._ptr(draws),
                                     asicp._ptr(theta)), "asicp_prop_sample")
        return theta
