"""Python binding of the surrogate network (C ABI in include/fargo_mlp.h).

Argument marshalling only: the forward pass, back-propagation, Adam and the
ensemble statistics run in the CUDA kernels of libfargo_b300.so.  Device
buffers are torch CUDA tensors (FP32, contiguous).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import FargoError, lib

_ready = False


def _lib():
    global _ready
    L = lib()
    if not _ready:
        vp = C.c_void_p
        L.fargo_mlp_create.argtypes = [C.POINTER(vp), C.POINTER(C.c_int), C.c_int, C.c_int, vp]
        L.fargo_mlp_destroy.argtypes = [vp]
        L.fargo_mlp_destroy.restype = None
        L.fargo_mlp_num_params.argtypes = [vp]
        L.fargo_mlp_num_params.restype = C.c_size_t
        for f in ("fargo_mlp_set_params", "fargo_mlp_get_params", "fargo_mlp_get_grads"):
            getattr(L, f).argtypes = [vp, vp, C.c_size_t]
        L.fargo_mlp_set_input_map.argtypes = [vp, vp, vp]
        L.fargo_mlp_set_output_map.argtypes = [vp, vp, vp]
        L.fargo_mlp_set_optimizer.argtypes = [vp, C.c_float, C.c_float, C.c_float, C.c_float]
        L.fargo_mlp_forward.argtypes = [vp, vp, C.c_int, vp]
        L.fargo_mlp_backward.argtypes = [vp, vp, vp, C.c_int, vp]
        L.fargo_mlp_adam.argtypes = [vp]
        L.fargo_mlp_train_step.argtypes = [vp, vp, vp, C.c_int, vp]
        L.fargo_mlp_ensemble.argtypes = [vp, C.c_int, C.c_int, C.c_int, vp, vp, vp]
        L.fargo_mlp_status.argtypes = [vp]
        _ready = True
    return L


def _check(rc, where):
    if rc != 0:
        raise FargoError(rc, where)


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class Mlp:
    """ReLU perceptron with bfloat16 tensor-core products (FP32 accumulate)."""

    def __init__(self, dims, max_batch, stream=None):
        self.dims = list(dims)
        arr = (C.c_int * len(dims))(*dims)
        h = C.c_void_p()
        _check(_lib().fargo_mlp_create(C.byref(h), arr, len(dims) - 1, max_batch, stream), "fargo_mlp_create")
        self.h = h
        self.max_batch = max_batch
        self.n = _lib().fargo_mlp_num_params(self.h)

    def close(self):
        if getattr(self, "h", None):
            _lib().fargo_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, vec):
        a = np.ascontiguousarray(vec, dtype=np.float32)
        _check(_lib().fargo_mlp_set_params(self.h, a.ctypes.data, a.size), "fargo_mlp_set_params")

    def get_params(self):
        a = np.empty(self.n, dtype=np.float32)
        _check(_lib().fargo_mlp_get_params(self.h, a.ctypes.data, a.size), "fargo_mlp_get_params")
        return a

    def get_grads(self):
        a = np.empty(self.n, dtype=np.float32)
        _check(_lib().fargo_mlp_get_grads(self.h, a.ctypes.data, a.size), "fargo_mlp_get_grads")
        return a

    def set_input_map(self, shift, scale):
        s = np.ascontiguousarray(shift, dtype=np.float32)
        c = np.ascontiguousarray(scale, dtype=np.float32)
        _check(_lib().fargo_mlp_set_input_map(self.h, s.ctypes.data, c.ctypes.data), "fargo_mlp_set_input_map")

    def set_output_map(self, shift, scale):
        s = np.ascontiguousarray(shift, dtype=np.float32)
        c = np.ascontiguousarray(scale, dtype=np.float32)
        _check(_lib().fargo_mlp_set_output_map(self.h, s.ctypes.data, c.ctypes.data), "fargo_mlp_set_output_map")

    def set_optimizer(self, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        _check(_lib().fargo_mlp_set_optimizer(self.h, lr, b1, b2, eps), "fargo_mlp_set_optimizer")

    def forward(self, x, out):
        _check(_lib().fargo_mlp_forward(self.h, _p(x), x.shape[0], _p(out)), "fargo_mlp_forward")
        return out

    def backward(self, x, t, loss=None):
        _check(_lib().fargo_mlp_backward(self.h, _p(x), _p(t), x.shape[0], _p(loss)), "fargo_mlp_backward")

    def adam(self):
        _check(_lib().fargo_mlp_adam(self.h), "fargo_mlp_adam")

    def status(self):
        """Synchronise; raises if a tensor-core product gave up waiting."""
        _check(_lib().fargo_mlp_status(self.h), "fargo_mlp_status")

    def train_step(self, x, t, loss=None):
        _check(_lib().fargo_mlp_train_step(self.h, _p(x), _p(t), x.shape[0], _p(loss)), "fargo_mlp_train_step")


def ensemble(ys, mean, spread, stream=None):
    """ys: (k, batch, n) device tensor; fills mean (batch, n) and spread (batch)."""
    k, b, n = ys.shape
    _check(_lib().fargo_mlp_ensemble(_p(ys), k, b, n, _p(mean), _p(spread), stream), "fargo_mlp_ensemble")
