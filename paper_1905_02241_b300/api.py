"""Object wrapper over the C ABI for torch tensors (marshalling only).

    ctx = Context(device=0, precision=NMODL_FP64)
    m = Mechanism(ctx, NMODL_CNEXP, node_index, n_nodes, params)
    m.init(v); ctx.step([m], dt, cm, v, rhs, d, nsteps)

Tensors must be contiguous and on the context's device (float64 for v, rhs,
d and states).  Every call enqueues on the context's stream (by default a
dedicated stream, so that windows can be replayed from CUDA graphs); each
enqueuing call is ordered after torch's current stream and torch's current
stream after it, so tensors may be produced and consumed with torch freely.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _lib
from ._lib import (NMODL_CACUM, NMODL_CNEXP, NMODL_FP64, NMODL_HH, NMODL_ION_CA,
                   NMODL_ION_K, NMODL_ION_NA, NMODL_ION_NONE, NMODL_KIN3, NMODL_KIN9,
                   NMODL_MIXED, NmodlError)

__all__ = ["Context", "Mechanism", "NmodlError", "NMODL_HH", "NMODL_CNEXP",
           "NMODL_KIN9", "NMODL_KIN3", "NMODL_CACUM", "NMODL_FP64", "NMODL_MIXED",
           "NMODL_ION_NONE", "NMODL_ION_NA", "NMODL_ION_K", "NMODL_ION_CA"]


def _dptr(t: torch.Tensor, dtype=torch.float64, device=None) -> int:
    if not isinstance(t, torch.Tensor):
        raise TypeError("expected a torch.Tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise ValueError(f"expected a contiguous {dtype} tensor")
    if device is not None and (t.device.type != "cuda" or t.device.index != device):
        raise ValueError(f"tensor must live on cuda:{device}")
    return t.data_ptr()


class Context:
    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None,
                 **options):
        self.device = int(device)
        self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
        opt = _lib.nmodl_options_default()
        for k, v in options.items():
            setattr(opt, k, v)
        self.options = opt
        self.handle = _lib.nmodl_ctx_create(self.device, self.stream.cuda_stream, opt)

    def enter(self) -> None:
        self.stream.wait_stream(torch.cuda.current_stream(self.device))

    def leave(self) -> None:
        torch.cuda.current_stream(self.device).wait_stream(self.stream)

    def set_options(self, **options) -> None:
        for k, v in options.items():
            setattr(self.options, k, v)
        _lib.nmodl_ctx_set_options(self.handle, self.options)

    def sync(self) -> int:
        return _lib.nmodl_sync(self.handle)

    def check(self) -> None:
        s = self.sync()
        if s:
            raise NmodlError(s, "device")

    def step(self, mechs, dt, cm, v, rhs, d, nsteps: int) -> None:
        self.enter()
        _lib.nmodl_step(self.handle, [m.handle for m in mechs], dt, cm,
                        _dptr(v, device=self.device), _dptr(rhs, device=self.device),
                        _dptr(d, device=self.device), nsteps)
        self.leave()

    def set_ions(self, ina=None, ik=None, ica=None) -> None:
        """Register per-node ion current arrays (float64 device tensors of
        n_nodes; None leaves that ion unrecorded; all None unregisters).
        The tensors must stay alive while registered."""
        ts = [t for t in (ina, ik, ica) if t is not None]
        n = ts[0].numel() if ts else 0
        if any(t.numel() != n for t in ts):
            raise ValueError("ion arrays must have equal lengths")
        ptr = [0 if t is None else _dptr(t, device=self.device) for t in (ina, ik, ica)]
        self.enter()
        _lib.nmodl_ctx_set_ions(self.handle, n, *ptr)
        self.leave()
        self._ions = (ina, ik, ica)

    def plan(self, mechs) -> dict:
        return _lib.nmodl_plan_describe(self.handle, [m.handle for m in mechs])

    def close(self) -> None:
        if self.handle:
            _lib.nmodl_ctx_destroy(self.handle)
            self.handle = 0


class Mechanism:
    def __init__(self, ctx: Context, mtype: int, node_index, n_nodes: int, params,
                 ion: int = NMODL_ION_NONE):
        self.ctx = ctx
        self.type = int(mtype)
        self.n_nodes = int(n_nodes)
        p = np.ascontiguousarray(params, dtype=np.float64)
        if isinstance(node_index, torch.Tensor):
            ni = node_index.contiguous()
            if ni.dtype != torch.int32:
                raise ValueError("node_index must be int32")
            ptr = ni.data_ptr()
            n = ni.numel()
        else:
            ni = np.ascontiguousarray(node_index, dtype=np.int32)
            ptr = ni.ctypes.data
            n = ni.size
        self.n = int(n)
        ctx.enter()
        self.handle = _lib.nmodl_mech_create(ctx.handle, self.type, self.n,
                                             ptr if n else 0, self.n_nodes,
                                             p.ctypes.data, p.size)
        ctx.leave()
        self.n_states = _lib.nmodl_mech_n_states(self.handle)
        self.ion = NMODL_ION_NONE
        if ion != NMODL_ION_NONE:
            self.set_ion(ion)

    def set_ion(self, ion: int) -> None:
        """Tag the mechanism's whole current as the current of ion `ion`."""
        _lib.nmodl_mech_set_ion(self.handle, ion)
        self.ion = int(ion)

    def init(self, v: torch.Tensor) -> None:
        self.ctx.enter()
        _lib.nmodl_init(self.handle, _dptr(v, device=self.ctx.device))
        self.ctx.leave()

    def state(self, dt: float, v: torch.Tensor) -> None:
        self.ctx.enter()
        _lib.nmodl_state(self.handle, dt, _dptr(v, device=self.ctx.device))
        self.ctx.leave()

    def cur(self, v, rhs, d) -> None:
        dev = self.ctx.device
        self.ctx.enter()
        _lib.nmodl_cur(self.handle, _dptr(v, device=dev), _dptr(rhs, device=dev),
                       _dptr(d, device=dev))
        self.ctx.leave()

    def get_state(self, k: int, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n, dtype=torch.float64, device=f"cuda:{self.ctx.device}")
        self.ctx.enter()
        _lib.nmodl_get_state(self.handle, k, _dptr(out) if self.n else 0)
        self.ctx.leave()
        return out

    def set_state(self, k: int, x: torch.Tensor) -> None:
        self.ctx.enter()
        _lib.nmodl_set_state(self.handle, k, _dptr(x) if self.n else 0)
        self.ctx.leave()

    def states(self) -> torch.Tensor:
        """All states as a (n_states, n) float64 device tensor (copy)."""
        out = torch.empty((self.n_states, self.n), dtype=torch.float64,
                          device=f"cuda:{self.ctx.device}")
        for k in range(self.n_states):
            self.get_state(k, out[k])
        return out

    def set_states(self, x: torch.Tensor) -> None:
        x = x.contiguous()
        for k in range(self.n_states):
            self.set_state(k, x[k].contiguous())

    def stats(self) -> dict:
        s = _lib.nmodl_stats(self.handle)
        return {k: getattr(s, k) for k, _ in s._fields_ if k != "reserved"}

    def close(self) -> None:
        if self.handle:
            _lib.nmodl_mech_destroy(self.handle)
            self.handle = 0


class Cable:
    """Cells of compartments with a tree morphology (nmodl_cable_*)."""

    def __init__(self, ctx: Context, parent, ga, gb):
        self.ctx = ctx
        p = np.ascontiguousarray(parent, dtype=np.int32)
        a = np.ascontiguousarray(ga, dtype=np.float64)
        b = np.ascontiguousarray(gb, dtype=np.float64)
        self.n_nodes = p.size
        ctx.enter()
        self.handle = _lib.nmodl_cable_create(ctx.handle, p.size, p.ctypes.data, a.ctypes.data,
                                              b.ctypes.data)
        self.n_cells = _lib.nmodl_cable_n_cells(self.handle)

    def step(self, mechs, dt, cm, v, rhs, d, nsteps: int) -> None:
        dev = self.ctx.device
        self.ctx.enter()
        _lib.nmodl_step_cable(self.ctx.handle, self.handle, [m.handle for m in mechs], dt, cm,
                              _dptr(v, device=dev), _dptr(rhs, device=dev),
                              _dptr(d, device=dev), nsteps)
        self.ctx.leave()

    def close(self) -> None:
        if self.handle:
            _lib.nmodl_cable_destroy(self.handle)
            self.handle = 0
