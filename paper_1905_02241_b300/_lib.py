"""ctypes binding of libnmodl_b300.so -- argument marshalling only.

Every function keeps the C name (nmodl_*) and takes plain integers for
pointers; tensors are passed by their data_ptr().  A non-zero status raises
NmodlError.  There is no fallback: if the shared library is absent the
import fails.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libnmodl_b300.so")

NMODL_OK = 0
NMODL_HH, NMODL_CNEXP, NMODL_KIN9, NMODL_CACUM, NMODL_KIN3 = 1, 2, 3, 4, 5
NMODL_ION_NONE, NMODL_ION_NA, NMODL_ION_K, NMODL_ION_CA = 0, 1, 2, 3
NMODL_FP64, NMODL_MIXED = 0, 1
ERRORS = {
    -1: "NMODL_ERR_ARG", -2: "NMODL_ERR_UNSORTED", -3: "NMODL_ERR_OOM",
    -4: "NMODL_ERR_CUDA", -5: "NMODL_ERR_NONFINITE", -6: "NMODL_ERR_NOCONV",
    -7: "NMODL_ERR_TIMEOUT", -8: "NMODL_ERR_RANGE", -9: "NMODL_ERR_UNSUPPORTED",
    -10: "NMODL_ERR_TOO_LARGE",
}


class NmodlError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        super().__init__(f"{what}: {ERRORS.get(status, status)} "
                         f"({_strerror(status)})")


class nmodl_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("newton_max_iter", ctypes.c_int32),
                ("newton_tol", ctypes.c_double), ("ir_max", ctypes.c_int32),
                ("window", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("autotune", ctypes.c_int32), ("clamp_v", ctypes.c_int32),
                ("tile_smem", ctypes.c_int32), ("block", ctypes.c_int32),
                ("cnexp_pade", ctypes.c_int32), ("no_fuse", ctypes.c_int32),
                ("reserved", ctypes.c_int32 * 3)]


class nmodl_stats_t(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("newton_iters", ctypes.c_int64),
                ("newton_max", ctypes.c_int64), ("nonconverged", ctypes.c_int64),
                ("fallback", ctypes.c_int64), ("surrogate_calls", ctypes.c_int64),
                ("reserved", ctypes.c_int64 * 2)]


if not os.path.exists(LIB_PATH):
    raise ImportError(f"{LIB_PATH} is missing: build it with "
                      "`python -m paper_1905_02241_b300.build`")

lib = ctypes.CDLL(LIB_PATH)
_vp, _i32, _i64, _d = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double
_P = ctypes.POINTER

_SIGS = {
    "nmodl_version": (_i32, []),
    "nmodl_strerror": (ctypes.c_char_p, [_i32]),
    "nmodl_options_default": (_i32, [_P(nmodl_options)]),
    "nmodl_ctx_create": (_i32, [_i32, _vp, _P(nmodl_options), _P(_vp)]),
    "nmodl_ctx_set_options": (_i32, [_vp, _P(nmodl_options)]),
    "nmodl_sync": (_i32, [_vp]),
    "nmodl_ctx_destroy": (None, [_vp]),
    "nmodl_mech_create": (_i32, [_vp, _i32, _i64, _vp, _i64, _vp, _i64, _P(_vp)]),
    "nmodl_mech_destroy": (None, [_vp]),
    "nmodl_mech_n_states": (_i32, [_vp]),
    "nmodl_init": (_i32, [_vp, _vp]),
    "nmodl_state": (_i32, [_vp, _d, _vp]),
    "nmodl_cur": (_i32, [_vp, _vp, _vp, _vp]),
    "nmodl_step": (_i32, [_vp, _vp, _i32, _d, _d, _vp, _vp, _vp, _i32]),
    "nmodl_get_state": (_i32, [_vp, _i32, _vp]),
    "nmodl_set_state": (_i32, [_vp, _i32, _vp]),
    "nmodl_stats": (_i32, [_vp, _P(nmodl_stats_t)]),
    "nmodl_probe_peak": (_i32, [_i32, _i32, _P(_d)]),
    "nmodl_probe_wait": (_i32, [_vp, _i32]),
    "nmodl_cur_noalloc": (_i32, [_i32, _vp, _i32, _i64, _vp, _i64, _vp, _i64, _vp,
                                 _i64, _vp, _vp, _vp]),
    "nmodl_cur_noalloc_max_instances": (_i64, []),
    "nmodl_surrogate_n_params": (_i32, []),
    "nmodl_surrogate_create": (_i32, [_vp, _i64, _vp, _i32, _P(_vp)]),
    "nmodl_surrogate_destroy": (None, [_vp]),
    "nmodl_surrogate_set_weights": (_i32, [_vp, _vp]),
    "nmodl_surrogate_get_weights": (_i32, [_vp, _vp]),
    "nmodl_surrogate_forward": (_i32, [_vp, _i64, _vp, _vp]),
    "nmodl_surrogate_loss_grad": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp]),
    "nmodl_surrogate_train_step": (_i32, [_vp, _i64, _vp, _vp, ctypes.c_float, _vp]),
    "nmodl_surrogate_fit": (_i32, [_vp, _i64, _vp, _vp, _i64, _i32, ctypes.c_float,
                                   ctypes.c_float, _vp]),
    "nmodl_surrogate_make_pairs": (_i32, [_vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _vp, _vp]),
    "nmodl_kin9_solve": (_i32, [_vp, _i64, _vp, _vp, _vp, _vp, _i64]),
    "nmodl_mech_attach_surrogate": (_i32, [_vp, _vp, _d]),
    "nmodl_plan_describe": (_i32, [_vp, _vp, _i32, _vp]),
    "nmodl_math_eval": (_i32, [_i32, _i64, _vp, _vp, _vp]),
    "nmodl_cable_create": (_i32, [_vp, _i64, _vp, _vp, _vp, _P(_vp)]),
    "nmodl_cable_destroy": (None, [_vp]),
    "nmodl_cable_n_cells": (_i32, [_vp]),
    "nmodl_step_cable": (_i32, [_vp, _vp, _vp, _i32, _d, _d, _vp, _vp, _vp, _i32]),
    "nmodl_ctx_set_ions": (_i32, [_vp, _i64, _vp, _vp, _vp]),
    "nmodl_mech_set_ion": (_i32, [_vp, _i32]),
}
for _name, (_res, _args) in _SIGS.items():
    _f = getattr(lib, _name)
    _f.restype = _res
    _f.argtypes = _args

EXPORTED = tuple(_SIGS)


def _strerror(s: int) -> str:
    return lib.nmodl_strerror(int(s)).decode()


def _check(status: int, what: str) -> None:
    if status != NMODL_OK:
        raise NmodlError(status, what)


def nmodl_version() -> int:
    return lib.nmodl_version()


def nmodl_strerror(status: int) -> str:
    return _strerror(status)


def nmodl_options_default() -> nmodl_options:
    o = nmodl_options()
    _check(lib.nmodl_options_default(ctypes.byref(o)), "nmodl_options_default")
    return o


def nmodl_ctx_create(device: int, stream: int, opt: nmodl_options | None) -> int:
    h = _vp()
    _check(lib.nmodl_ctx_create(int(device), stream or None,
                                ctypes.byref(opt) if opt is not None else None,
                                ctypes.byref(h)), "nmodl_ctx_create")
    return h.value


def nmodl_ctx_set_options(ctx: int, opt: nmodl_options) -> None:
    _check(lib.nmodl_ctx_set_options(ctx, ctypes.byref(opt)), "nmodl_ctx_set_options")


def nmodl_sync(ctx: int) -> int:
    """Returns the latched device status (0 if none); raises on CUDA errors."""
    s = lib.nmodl_sync(ctx)
    if s == -4:
        _check(s, "nmodl_sync")
    return s


def nmodl_ctx_destroy(ctx: int) -> None:
    lib.nmodl_ctx_destroy(ctx)


def nmodl_mech_create(ctx: int, mtype: int, n_instances: int, node_index_ptr: int,
                      n_nodes: int, params_ptr: int, n_params: int) -> int:
    h = _vp()
    _check(lib.nmodl_mech_create(ctx, int(mtype), int(n_instances),
                                 node_index_ptr or None, int(n_nodes),
                                 params_ptr or None, int(n_params),
                                 ctypes.byref(h)), "nmodl_mech_create")
    return h.value


def nmodl_ctx_set_ions(ctx: int, n_nodes: int, ina_ptr: int, ik_ptr: int,
                       ica_ptr: int) -> None:
    _check(lib.nmodl_ctx_set_ions(ctx, int(n_nodes), ina_ptr or None, ik_ptr or None,
                                  ica_ptr or None), "nmodl_ctx_set_ions")


def nmodl_mech_set_ion(m: int, ion: int) -> None:
    _check(lib.nmodl_mech_set_ion(m, int(ion)), "nmodl_mech_set_ion")


def nmodl_mech_destroy(m: int) -> None:
    lib.nmodl_mech_destroy(m)


def nmodl_mech_n_states(m: int) -> int:
    return lib.nmodl_mech_n_states(m)


def nmodl_init(m: int, v_ptr: int) -> None:
    _check(lib.nmodl_init(m, v_ptr or None), "nmodl_init")


def nmodl_state(m: int, dt: float, v_ptr: int) -> None:
    _check(lib.nmodl_state(m, float(dt), v_ptr or None), "nmodl_state")


def nmodl_cur(m: int, v_ptr: int, rhs_ptr: int, d_ptr: int) -> None:
    _check(lib.nmodl_cur(m, v_ptr or None, rhs_ptr or None, d_ptr or None), "nmodl_cur")


def nmodl_step(ctx: int, mechs, dt: float, cm: float, v_ptr: int, rhs_ptr: int,
               d_ptr: int, nsteps: int) -> None:
    arr = (_vp * len(mechs))(*mechs)
    _check(lib.nmodl_step(ctx, ctypes.cast(arr, _vp), len(mechs), float(dt),
                          float(cm), v_ptr or None, rhs_ptr or None, d_ptr or None,
                          int(nsteps)), "nmodl_step")


def nmodl_get_state(m: int, k: int, out_ptr: int) -> None:
    _check(lib.nmodl_get_state(m, int(k), out_ptr or None), "nmodl_get_state")


def nmodl_set_state(m: int, k: int, in_ptr: int) -> None:
    _check(lib.nmodl_set_state(m, int(k), in_ptr or None), "nmodl_set_state")


def nmodl_stats(m: int) -> nmodl_stats_t:
    s = nmodl_stats_t()
    _check(lib.nmodl_stats(m, ctypes.byref(s)), "nmodl_stats")
    return s


def nmodl_probe_peak(device: int, kind: int) -> float:
    x = _d()
    _check(lib.nmodl_probe_peak(int(device), int(kind), ctypes.byref(x)), "nmodl_probe_peak")
    return x.value


def nmodl_cur_noalloc(device: int, stream: int, mtype: int, n_instances: int,
                      node_index_ptr: int, n_nodes: int, params_ptr: int, n_params: int,
                      states_ptr: int, stride: int, v_ptr: int, rhs_ptr: int,
                      d_ptr: int) -> None:
    _check(lib.nmodl_cur_noalloc(int(device), stream or None, int(mtype), int(n_instances),
                                 node_index_ptr or None, int(n_nodes), params_ptr or None,
                                 int(n_params), states_ptr or None, int(stride),
                                 v_ptr or None, rhs_ptr or None, d_ptr or None),
           "nmodl_cur_noalloc")


def nmodl_cur_noalloc_max_instances() -> int:
    return lib.nmodl_cur_noalloc_max_instances()


def nmodl_surrogate_n_params() -> int:
    return lib.nmodl_surrogate_n_params()


def nmodl_surrogate_create(ctx: int, max_batch: int, weights_ptr: int, scaled: int) -> int:
    h = _vp()
    _check(lib.nmodl_surrogate_create(ctx, int(max_batch), weights_ptr or None, int(scaled),
                                      ctypes.byref(h)), "nmodl_surrogate_create")
    return h.value


def nmodl_surrogate_destroy(s: int) -> None:
    lib.nmodl_surrogate_destroy(s)


def nmodl_surrogate_set_weights(s: int, w_ptr: int) -> None:
    _check(lib.nmodl_surrogate_set_weights(s, w_ptr), "nmodl_surrogate_set_weights")


def nmodl_surrogate_get_weights(s: int, w_ptr: int) -> None:
    _check(lib.nmodl_surrogate_get_weights(s, w_ptr), "nmodl_surrogate_get_weights")


def nmodl_surrogate_forward(s: int, n: int, X_ptr: int, Y_ptr: int) -> None:
    _check(lib.nmodl_surrogate_forward(s, int(n), X_ptr, Y_ptr), "nmodl_surrogate_forward")


def nmodl_surrogate_loss_grad(s: int, n: int, X_ptr: int, T_ptr: int, grad_ptr: int,
                              loss_ptr: int) -> None:
    _check(lib.nmodl_surrogate_loss_grad(s, int(n), X_ptr, T_ptr, grad_ptr or None,
                                         loss_ptr or None), "nmodl_surrogate_loss_grad")


def nmodl_surrogate_train_step(s: int, n: int, X_ptr: int, T_ptr: int, lr: float,
                               loss_ptr: int) -> None:
    _check(lib.nmodl_surrogate_train_step(s, int(n), X_ptr, T_ptr, float(lr), loss_ptr or None),
           "nmodl_surrogate_train_step")


def nmodl_surrogate_make_pairs(s: int, kin: int, n: int, v_ptr: int, dt_ptr: int, x_ptr: int,
                               y_ptr: int, stride: int, X_ptr: int, T_ptr: int) -> None:
    _check(lib.nmodl_surrogate_make_pairs(s, kin, int(n), v_ptr, dt_ptr, x_ptr, y_ptr,
                                          int(stride), X_ptr, T_ptr),
           "nmodl_surrogate_make_pairs")


def nmodl_kin9_solve(kin: int, n: int, v_ptr: int, dt_ptr: int, x_ptr: int, y_ptr: int,
                     stride: int) -> None:
    _check(lib.nmodl_kin9_solve(kin, int(n), v_ptr, dt_ptr, x_ptr, y_ptr, int(stride)),
           "nmodl_kin9_solve")


def nmodl_mech_attach_surrogate(m: int, s: int, tol: float) -> None:
    _check(lib.nmodl_mech_attach_surrogate(m, s or None, float(tol)),
           "nmodl_mech_attach_surrogate")


def nmodl_plan_describe(ctx: int, mechs) -> dict:
    arr = (_vp * len(mechs))(*mechs)
    out = (ctypes.c_int64 * 6)()
    _check(lib.nmodl_plan_describe(ctx, ctypes.cast(arr, _vp), len(mechs),
                                   ctypes.cast(out, _vp)), "nmodl_plan_describe")
    form = {0: "launches", 1: "tiles", 2: "hh_gate_warps", 3: "surrogate_step"}[int(out[0])]
    return dict(fused=bool(out[0]), form=form, tiles=int(out[1]), block=int(out[2]),
                smem=int(out[3]), persistent=bool(out[4]), tile_budget=int(out[5]))


def nmodl_math_eval(fn: int, n: int, x_ptr: int, y_ptr: int, stream: int) -> None:
    _check(lib.nmodl_math_eval(int(fn), int(n), x_ptr, y_ptr, stream or None), "nmodl_math_eval")


def nmodl_cable_create(ctx: int, n_nodes: int, parent_ptr: int, ga_ptr: int, gb_ptr: int) -> int:
    h = _vp()
    _check(lib.nmodl_cable_create(ctx, int(n_nodes), parent_ptr, ga_ptr, gb_ptr, ctypes.byref(h)),
           "nmodl_cable_create")
    return h.value


def nmodl_cable_destroy(cb: int) -> None:
    lib.nmodl_cable_destroy(cb)


def nmodl_cable_n_cells(cb: int) -> int:
    return lib.nmodl_cable_n_cells(cb)


def nmodl_step_cable(ctx: int, cb: int, mechs, dt: float, cm: float, v_ptr: int, rhs_ptr: int,
                     d_ptr: int, nsteps: int) -> None:
    arr = (_vp * len(mechs))(*mechs)
    _check(lib.nmodl_step_cable(ctx, cb, ctypes.cast(arr, _vp), len(mechs), float(dt),
                                float(cm), v_ptr, rhs_ptr, d_ptr, int(nsteps)), "nmodl_step_cable")


def nmodl_surrogate_fit(sur: int, n: int, X_ptr: int, T_ptr: int, batch: int, epochs: int,
                        lr: float, lr_min: float, loss_ptr: int) -> None:
    _check(lib.nmodl_surrogate_fit(sur, int(n), X_ptr, T_ptr, int(batch), int(epochs),
                                   float(lr), float(lr_min), loss_ptr), "nmodl_surrogate_fit")


def nmodl_probe_wait(ctx, polls: int) -> None:
    _check(lib.nmodl_probe_wait(ctx, int(polls)), "nmodl_probe_wait")
