"""Kinetic surrogate: Newton-generated training pairs and the training loop
(orchestration over the C ABI; every arithmetic step runs in the library's
kernels).

    sur = Surrogate(ctx)                       # zero weights
    sur.set_weights(w)                         # or W.mlp_init(...)
    X, T = make_training_pairs(ctx, sur, kin_params, n, seed)
    sur.fit(X, T, epochs=..., batch=8192)
    mech.attach_surrogate(sur, tol=1e-4)       # nmodl_state uses it
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import _lib
from . import workloads as W
from .api import Context, Mechanism


class Surrogate:
    N_PARAMS = _lib.nmodl_surrogate_n_params()

    def __init__(self, ctx: Context, max_batch: int = 8192, weights=None, scaled: bool = True):
        self.ctx = ctx
        self.max_batch = int(max_batch)
        w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
        self.handle = _lib.nmodl_surrogate_create(ctx.handle, self.max_batch,
                                                  w.ctypes.data if w is not None else 0,
                                                  int(bool(scaled)))
        self.scaled = bool(scaled)

    @staticmethod
    def pack(Ws, bs) -> np.ndarray:
        """Public parameter vector from per-layer [out][in] weights and biases."""
        parts = []
        for Wl, bl in zip(Ws, bs):
            parts += [np.asarray(Wl, np.float32).ravel(), np.asarray(bl, np.float32).ravel()]
        return np.ascontiguousarray(np.concatenate(parts))

    @staticmethod
    def unpack(w, widths=(11, 128, 128, 128, 9)):
        Ws, bs, o = [], [], 0
        for li in range(len(widths) - 1):
            fi, fo = widths[li], widths[li + 1]
            Ws.append(np.asarray(w[o:o + fi * fo], np.float64).reshape(fo, fi))
            o += fi * fo
            bs.append(np.asarray(w[o:o + fo], np.float64))
            o += fo
        return Ws, bs

    def set_weights(self, w) -> None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        assert w.size == self.N_PARAMS
        self.ctx.enter()
        _lib.nmodl_surrogate_set_weights(self.handle, w.ctypes.data)
        self.ctx.leave()

    def get_weights(self) -> np.ndarray:
        w = np.zeros(self.N_PARAMS, dtype=np.float32)
        self.ctx.enter()
        _lib.nmodl_surrogate_get_weights(self.handle, w.ctypes.data)
        self.ctx.leave()
        return w

    def forward(self, X: torch.Tensor) -> torch.Tensor:
        n = X.shape[0]
        Y = torch.empty((n, 9), dtype=torch.float32, device=X.device)
        self.ctx.enter()
        _lib.nmodl_surrogate_forward(self.handle, n, X.data_ptr(), Y.data_ptr())
        self.ctx.leave()
        return Y

    def loss_grad(self, X: torch.Tensor, T: torch.Tensor):
        g = np.zeros(self.N_PARAMS, dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self.ctx.enter()
        _lib.nmodl_surrogate_loss_grad(self.handle, X.shape[0], X.data_ptr(), T.data_ptr(),
                                       g.ctypes.data, loss.ctypes.data)
        self.ctx.leave()
        return float(loss[0]), g

    def fit(self, X: torch.Tensor, T: torch.Tensor, epochs: int = 20, batch: int = 8192,
            lr: float = 2e-3, lr_min: float = 1e-5, log_every: int = 0):
        """Adam over mini-batches in the (already random) order of the rows,
        learning rate on a cosine schedule from lr to lr_min (the library
        replays one captured optimiser step per minibatch).  Returns the mean
        loss of each epoch."""
        n = X.shape[0] // batch * batch
        steps_per_epoch = n // batch
        total = epochs * steps_per_epoch
        loss_dev = torch.zeros(total, dtype=torch.float32, device=X.device)
        self.ctx.enter()
        _lib.nmodl_surrogate_fit(self.handle, n, X.data_ptr(), T.data_ptr(), batch, epochs,
                                 lr, lr_min, loss_dev.data_ptr())
        self.ctx.leave()
        losses = loss_dev.view(epochs, steps_per_epoch).mean(dim=1).cpu().numpy()
        return losses

    def close(self) -> None:
        if self.handle:
            _lib.nmodl_surrogate_destroy(self.handle)
            self.handle = 0


def attach(mech: Mechanism, sur: Surrogate | None, tol: float = 1e-4) -> None:
    _lib.nmodl_mech_attach_surrogate(mech.handle, sur.handle if sur else 0, tol)


def newton_pairs(ctx: Context, kin_params, n: int, seed: int = 6):
    """(v, dt, x, y): n sampled inputs and their FP64 Newton implicit Euler
    step, on the device (x, y SoA (9, n))."""
    v, dt, x, lam = W.surrogate_samples(n, seed)
    dev = f"cuda:{ctx.device}"
    v_t = torch.tensor(v, device=dev)
    dt_t = torch.tensor(dt, device=dev)
    kin = Mechanism(ctx, W.TYPE_KIN9, np.arange(n, dtype=np.int32), n, kin_params)
    try:
        kin.init(v_t)                                   # stationary distributions
        pi = kin.states()
        lam_t = torch.tensor(lam, device=dev)
        x_t = lam_t * pi + (1.0 - lam_t) * torch.tensor(x, device=dev)
        x_t = x_t.contiguous()
        y_t = torch.empty_like(x_t)
        ctx.enter()
        _lib.nmodl_kin9_solve(kin.handle, n, v_t.data_ptr(), dt_t.data_ptr(), x_t.data_ptr(),
                              y_t.data_ptr(), n)
        ctx.leave()
        assert ctx.sync() == 0
    finally:
        kin.close()
    return v_t, dt_t, x_t, y_t


def make_training_pairs(ctx: Context, sur: Surrogate, kin_params, n: int, seed: int = 6):
    """Normalised inputs X [n][11] and targets T [n][9] (FP32, device)."""
    v_t, dt_t, x_t, y_t = newton_pairs(ctx, kin_params, n, seed)
    kin = Mechanism(ctx, W.TYPE_KIN9, np.zeros(1, dtype=np.int32), 1, kin_params)
    X = torch.empty((n, 11), dtype=torch.float32, device=v_t.device)
    T = torch.empty((n, 9), dtype=torch.float32, device=v_t.device)
    ctx.enter()
    _lib.nmodl_surrogate_make_pairs(sur.handle, kin.handle, n, v_t.data_ptr(), dt_t.data_ptr(),
                                    x_t.data_ptr(), y_t.data_ptr(), n, X.data_ptr(), T.data_ptr())
    ctx.leave()
    assert ctx.sync() == 0
    kin.close()
    return X, T
