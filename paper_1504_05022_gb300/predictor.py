"""Learned preallocation: row features, the MLP kernels and a device predictor.

Thin wrappers over the C ABI (spgemm_row_features, spgemm_mlp_*,
spgemm_predictor_*); every computation runs in the library's CUDA kernels."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np
import torch

from . import _lib
from .spgemm import CSR

WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "predictor_weights.json")


def _s(stream):
    return ctypes.c_void_p((stream or torch.cuda.current_stream()).cuda_stream)


def row_features(A: CSR, B: CSR, stream=None) -> torch.Tensor:
    """[m, 8] float32 features of the rows of C = A*B (computed on the GPU)."""
    L = _lib.load()
    X = torch.empty((A.nrows, _lib.MLP_FEATURES), dtype=torch.float32, device=A.val.device)
    a, b = A._c_in(), B._c_in()
    _lib.check(L.spgemm_row_features(ctypes.byref(a), ctypes.byref(b), ctypes.c_void_p(X.data_ptr()), _s(stream)),
               "spgemm_row_features")
    return X


def mlp_forward(params: torch.Tensor, X: torch.Tensor, stream=None) -> torch.Tensor:
    L = _lib.load()
    out = torch.empty((X.shape[0], _lib.MLP_CLASSES + 1), dtype=torch.float32, device=X.device)
    _lib.check(L.spgemm_mlp_forward(ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(X.data_ptr()), X.shape[0],
                                    ctypes.c_void_p(out.data_ptr()), _s(stream)), "spgemm_mlp_forward")
    return out


class Trainer:
    """Adam on the device with the library's gradient kernels."""

    def __init__(self, params: torch.Tensor, lr: float = 3e-3):
        self.L = _lib.load()
        self.params = params.contiguous()
        dev = params.device
        self.grad = torch.zeros(_lib.MLP_NUM_PARAMS, dtype=torch.float32, device=dev)
        self.m = torch.zeros_like(self.grad)
        self.v = torch.zeros_like(self.grad)
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.work = None
        self.lr = lr
        self.t = 0

    def loss_grad(self, X, cls, y, stream=None):
        n = X.shape[0]
        need = int(self.L.spgemm_mlp_work_floats(n))
        if self.work is None or self.work.numel() < need:
            self.work = torch.empty(max(need, 1), dtype=torch.float32, device=X.device)
        _lib.check(self.L.spgemm_mlp_loss_grad(
            ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(cls.data_ptr()),
            ctypes.c_void_p(y.data_ptr()), n, ctypes.c_void_p(self.work.data_ptr()),
            ctypes.c_void_p(self.grad.data_ptr()), ctypes.c_void_p(self.loss.data_ptr()), _s(stream)),
            "spgemm_mlp_loss_grad")
        return self.loss, self.grad

    def step(self, X, cls, y, lr=None, stream=None):
        self.loss_grad(X, cls, y, stream)
        self.t += 1
        _lib.check(self.L.spgemm_mlp_adam(
            ctypes.c_void_p(self.params.data_ptr()), ctypes.c_void_p(self.grad.data_ptr()),
            ctypes.c_void_p(self.m.data_ptr()), ctypes.c_void_p(self.v.data_ptr()), self.t,
            float(lr if lr is not None else self.lr), 1.0 / max(1, X.shape[0]), _s(stream)), "spgemm_mlp_adam")
        return self.loss


class Predictor:
    """Device copy of a parameter vector, usable as opts.predictor (alloc_policy='learned')."""

    def __init__(self, params, margin: float = 1.0, dtype: str = "f64"):
        L = self.L = _lib.load(dtype=dtype)
        self.dtype = dtype  # the value type of the plans it serves ("f64" or "f32")
        host = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
        if host.size != _lib.MLP_NUM_TOTAL:
            raise ValueError(f"expected {_lib.MLP_NUM_TOTAL} parameters, got {host.size}")
        h = ctypes.c_void_p()
        _lib.check(L.spgemm_predictor_create(host.ctypes.data_as(ctypes.c_void_p), host.size, ctypes.byref(h)),
                   "spgemm_predictor_create")
        self.handle = h.value
        self.margin = float(margin)
        self.params = host

    def opts(self) -> dict:
        """Plan options for the learned policy.  The entry "predictor" is this object itself, so
        every Plan made from these options keeps the device weights alive."""
        return {"alloc_policy": "learned", "predictor": self, "predictor_margin": self.margin}

    def __del__(self):
        try:
            if self.handle:
                self.L.spgemm_predictor_free(ctypes.c_void_p(self.handle))
                self.handle = None
        except Exception:
            pass

    @classmethod
    def load(cls, path: str = WEIGHTS, margin: float | None = None, dtype: str = "f64") -> "Predictor":
        with open(path) as f:
            d = json.load(f)
        return cls(np.array(d["params"], dtype=np.float32), d.get("margin", 1.0) if margin is None else margin,
                   dtype=dtype)
