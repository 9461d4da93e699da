"""Python face of the FP64 CPU oracle (test infrastructure only).

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference
legs may import this module.  The mechanism routines live in
nmodl_oracle.c (plain C, libm, FP64) and are reached through ctypes; the
surrogate network and the simplex projection are plain numpy below.

Citations are to the paper's sections (arXiv 1905.02241): Section 5.2 for
cnexp, implicit Euler, sparse/derivimplicit and the analytic conductance,
Section 5.3 for the LU and Newton solves, Section 3 for BREAKPOINT.

Parity pins: every function here is checked by tests/test_oracle_pins.py
against closed forms, invariants, an independent root find, least squares,
high-precision evaluation or brute-force RK4 (see that file's docstring).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "nmodl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

TYPE_HH, TYPE_CNEXP, TYPE_KIN9, TYPE_CACUM, TYPE_KIN3 = 1, 2, 3, 4, 5
ION_NONE, ION_NA, ION_K, ION_CA = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile nmodl_oracle.c into liboracle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
               "-shared", "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
        vp = ctypes.c_void_p
        L.orc_vtrap.restype = d
        L.orc_vtrap.argtypes = [d, d]
        L.orc_rate.restype = d
        L.orc_rate.argtypes = [ctypes.c_int, d, d, d, d]
        L.orc_hh_rates.argtypes = [vp, d, vp, vp]
        L.orc_cnexp_rates.argtypes = [vp, ctypes.c_int, d, vp, vp]
        L.orc_mech_init.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp]
        L.orc_mech_state.argtypes = [ctypes.c_int, i64, vp, vp, vp, d, vp, d,
                                     ctypes.c_int, vp]
        L.orc_mech_cur.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, vp]
        L.orc_mech_currents.argtypes = [ctypes.c_int, i64, vp, vp, vp, vp, vp, vp]
        L.orc_kin9_matrix.argtypes = [vp, d, vp]
        L.orc_kin9_stationary.restype = ctypes.c_int
        L.orc_kin9_stationary.argtypes = [vp, d, vp]
        L.orc_kin9_state.argtypes = [i64, vp, vp, vp, d, vp, d, ctypes.c_int,
                                     vp, vp]
        L.orc_kin9_newton.restype = ctypes.c_int
        L.orc_kin9_newton.argtypes = [vp, d, vp, vp, d, ctypes.c_int, vp]
        L.orc_lu_pp.restype = ctypes.c_int
        L.orc_lu_pp.argtypes = [ctypes.c_int, vp, vp]
        L.orc_lu_solve.argtypes = [ctypes.c_int, vp, vp, vp, vp]
        L.orc_step.argtypes = [ctypes.c_int, vp, i64, d, d, vp, vp, vp,
                               ctypes.c_int, ctypes.c_int, d, ctypes.c_int]
        L.orc_step_cable.argtypes = [ctypes.c_int, vp, i64, vp, vp, vp, d, d, vp, vp,
                                     vp, ctypes.c_int, d, ctypes.c_int]
        L.orc_cnexp_factor.restype = d
        L.orc_cnexp_factor.argtypes = [d]
        L.orc_kin3_matrix.argtypes = [vp, d, vp]
        L.orc_kin_newton_n.restype = ctypes.c_int
        L.orc_kin_newton_n.argtypes = [ctypes.c_int, vp, d, vp, vp, d, ctypes.c_int]
        L.orc_kin_stationary_n.restype = ctypes.c_int
        L.orc_kin_stationary_n.argtypes = [ctypes.c_int, vp, vp]
        L.orc_cacum_newton.restype = ctypes.c_int
        L.orc_cacum_newton.argtypes = [vp, d, d, vp, vp, d, ctypes.c_int]
        L.orc_set_ion_read.argtypes = [ctypes.c_int, vp]
        L.orc_mech_ion_cur.argtypes = [ctypes.c_int, ctypes.c_int, i64, vp, vp, vp, vp, vp]
        L.orc_step_ions.argtypes = [ctypes.c_int, vp, i64, d, d, vp, vp, vp, vp,
                                    ctypes.c_int, ctypes.c_int, d, ctypes.c_int]
        _ = (P, i32)
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


NEWTON_TOL = 1e-14
NEWTON_MAX_ITER = 8


def n_states(mtype: int, params: np.ndarray) -> int:
    if mtype == TYPE_HH:
        return 3
    if mtype == TYPE_CNEXP:
        return int(params[0])
    if mtype == TYPE_KIN9:
        return 9
    if mtype == TYPE_CACUM:
        return 2
    if mtype == TYPE_KIN3:
        return 3
    raise ValueError(mtype)


# ------------------------------------------------------------------ scalars

def vtrap(x: float, y: float) -> float:
    return lib().orc_vtrap(float(x), float(y))


def rate(form: int, A: float, vh: float, k: float, v: float) -> float:
    return lib().orc_rate(int(form), float(A), float(vh), float(k), float(v))


def hh_rates(params, v: float):
    p = _f64(params)
    mi, mt = np.zeros(3), np.zeros(3)
    lib().orc_hh_rates(_p(p), float(v), _p(mi), _p(mt))
    return mi, mt


def cnexp_rates(params, g: int, v: float):
    p = _f64(params)
    mi, mt = np.zeros(1), np.zeros(1)
    lib().orc_cnexp_rates(_p(p), int(g), float(v), _p(mi), _p(mt))
    return float(mi[0]), float(mt[0])


def kin9_matrix(params, v: float) -> np.ndarray:
    p = _f64(params)
    A = np.zeros(81)
    lib().orc_kin9_matrix(_p(p), float(v), _p(A))
    return A.reshape(9, 9)


def kin9_stationary(params, v: float) -> np.ndarray:
    p = _f64(params)
    pi = np.zeros(9)
    rc = lib().orc_kin9_stationary(_p(p), float(v), _p(pi))
    if rc != 0:
        raise RuntimeError("singular stationary system")
    return pi


def lu_pp(M: np.ndarray):
    n = M.shape[0]
    LU = _f64(M).copy()
    perm = np.zeros(n, dtype=np.int32)
    sw = lib().orc_lu_pp(n, _p(LU), _p(perm))
    return LU, perm, sw


def lu_solve(LU, perm, b):
    n = LU.shape[0]
    x = np.zeros(n)
    lib().orc_lu_solve(n, _p(_f64(LU)), _p(_i32(perm)), _p(_f64(b)), _p(x))
    return x


def kin9_newton(A, dt, x, tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    y = np.zeros(9)
    sw = np.zeros(1, dtype=np.int32)
    it = lib().orc_kin9_newton(_p(_f64(A)), float(dt), _p(_f64(x)), _p(y),
                               float(tol), int(max_iter), _p(sw))
    return y, it, int(sw[0])


# ------------------------------------------------------------- mechanisms

def mech_init(mtype, params, node_index, v) -> np.ndarray:
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    n = ni.size
    s = np.zeros((n_states(mtype, p), n))
    lib().orc_mech_init(int(mtype), n, _p(ni), _p(vv), _p(p), _p(s))
    return s


def mech_state(mtype, params, node_index, v, states, dt,
               tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER, want_iters=False, ica=None):
    """Returns the updated SoA states (copy); optionally Newton iterations.
    ica: per-node calcium current read by the calcium accumulation type."""
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    s = _f64(states).copy()
    it = np.zeros(ni.size, dtype=np.int32)
    ic = None if ica is None else _f64(ica)
    L = lib()
    L.orc_set_ion_read(ION_CA, None if ic is None else _p(ic))
    try:
        L.orc_mech_state(int(mtype), ni.size, _p(ni), _p(vv), _p(p), float(dt),
                         _p(s), float(tol), int(max_iter), _p(it))
    finally:
        L.orc_set_ion_read(ION_CA, None)
    return (s, it) if want_iters else s


def kin9_state_swaps(params, node_index, v, states, dt):
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    s = _f64(states).copy()
    it = np.zeros(ni.size, dtype=np.int32)
    sw = np.zeros(1, dtype=np.int64)
    lib().orc_kin9_state(ni.size, _p(ni), _p(vv), _p(p), float(dt), _p(s),
                         NEWTON_TOL, NEWTON_MAX_ITER, _p(it), _p(sw))
    return s, it, int(sw[0])


def mech_cur(mtype, params, node_index, v, states, rhs, d):
    """Accumulates into copies of rhs and d; returns (rhs, d)."""
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    s = _f64(states)
    r, dd = _f64(rhs).copy(), _f64(d).copy()
    lib().orc_mech_cur(int(mtype), ni.size, _p(ni), _p(vv), _p(p), _p(s),
                       _p(r), _p(dd))
    return r, dd


def mech_currents(mtype, params, node_index, v, states):
    """Per-instance (i, g)."""
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    s = _f64(states)
    c, g = np.zeros(ni.size), np.zeros(ni.size)
    lib().orc_mech_currents(int(mtype), ni.size, _p(ni), _p(vv), _p(p), _p(s),
                            _p(c), _p(g))
    return c, g


def mech_ion_cur(mtype, params, node_index, v, states, n_nodes, ion=ION_NONE):
    """Per-node ion currents [4][n_nodes] (row 0 unused) of one mechanism:
    HH writes ina and ik, a CNEXP/KIN9/KIN3 mechanism tagged with ion writes
    its whole current to that ion."""
    p, ni, vv = _f64(params), _i32(node_index), _f64(v)
    s = _f64(states)
    out = np.zeros((4, int(n_nodes)))
    ptrs = (ctypes.c_void_p * 4)(None, *[out[k].ctypes.data for k in (1, 2, 3)])
    lib().orc_mech_ion_cur(int(mtype), int(ion), ni.size, _p(ni), _p(vv), _p(p), _p(s),
                           ctypes.cast(ptrs, ctypes.c_void_p))
    return out


def kin3_matrix(params, v: float) -> np.ndarray:
    A = np.zeros(9)
    lib().orc_kin3_matrix(_p(_f64(params)), float(v), _p(A))
    return A.reshape(3, 3)


def kin_newton_n(A, dt, x, tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    A = _f64(A)
    ns = A.shape[0]
    xx = _f64(x)
    y = np.zeros(ns)
    it = lib().orc_kin_newton_n(ns, _p(A), float(dt), _p(xx), _p(y), float(tol),
                                int(max_iter))
    return y, it


def kin_stationary_n(A) -> np.ndarray:
    A = _f64(A)
    pi = np.zeros(A.shape[0])
    if lib().orc_kin_stationary_n(A.shape[0], _p(A), _p(pi)) != 0:
        raise ArithmeticError("singular stationary system")
    return pi


def cacum_newton(params, dt, ica, x, tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    """One implicit Euler step of the calcium buffer; returns (y, iterations)."""
    xx, y = _f64(x), np.zeros(2)
    it = lib().orc_cacum_newton(_p(_f64(params)), float(dt), float(ica), _p(xx), _p(y),
                                float(tol), int(max_iter))
    return y, it


class _OrcMech(ctypes.Structure):
    _fields_ = [("type", ctypes.c_int32), ("ion", ctypes.c_int32),
                ("n", ctypes.c_int64), ("node_index", ctypes.c_void_p),
                ("params", ctypes.c_void_p), ("states", ctypes.c_void_p)]


def step(mechs, states, v, n_nodes, dt, cm=1.0, nsteps=1, clamp_v=False,
         tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    """nsteps steps of the whole network.

    mechs: list of dict(type, params, node_index); states: list of SoA arrays
    (copied).  Returns (v, rhs, d, states) after the last step.
    """
    keep = []
    arr = (_OrcMech * len(mechs))()
    out_states = []
    for k, m in enumerate(mechs):
        p, ni = _f64(m["params"]), _i32(m["node_index"])
        s = _f64(states[k]).copy()
        keep += [p, ni]
        out_states.append(s)
        arr[k].type = int(m["type"])
        arr[k].n = ni.size
        arr[k].node_index = ni.ctypes.data
        arr[k].params = p.ctypes.data
        arr[k].states = s.ctypes.data
    vv = _f64(v).copy()
    rhs, d = np.zeros(n_nodes), np.zeros(n_nodes)
    lib().orc_step(len(mechs), ctypes.cast(arr, ctypes.c_void_p), int(n_nodes),
                   float(dt), float(cm), _p(vv), _p(rhs), _p(d), int(nsteps),
                   int(bool(clamp_v)), float(tol), int(max_iter))
    return vv, rhs, d, out_states


# ------------------------------------------------- surrogate (plain numpy)
# The learned stand-in for the kinetic Newton solve: an MLP maps the
# normalised (v, dt, x) to an increment dx; x + dx is projected onto the
# probability simplex.  Normalisation: v_n = (v + 20)/80,
# dt_n = (dt - 0.03125)/0.01875, x unchanged.

V_SHIFT, V_SCALE = 20.0, 80.0
DT_SHIFT, DT_SCALE = 0.03125, 0.01875


def silu(z):
    return z / (1.0 + np.exp(-z))


def dsilu(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def surrogate_inputs(v, dt, x):
    """Columns of normalised inputs, shape (11, batch)."""
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    dt = np.broadcast_to(np.asarray(dt, dtype=np.float64), v.shape)
    return np.vstack([(v + V_SHIFT) / V_SCALE, (dt - DT_SHIFT) / DT_SCALE,
                      np.asarray(x, dtype=np.float64).reshape(9, -1)])


def mlp_forward(Ws, bs, X):
    """X: (11, batch).  Returns (out (9, batch), cache of pre-activations)."""
    h = X
    zs, hs = [], [X]
    for li, (W, b) in enumerate(zip(Ws, bs)):
        z = W @ h + b[:, None]
        zs.append(z)
        h = silu(z) if li < len(Ws) - 1 else z
        hs.append(h)
    return h, (zs, hs)


def mlp_loss_grad(Ws, bs, X, T):
    """Mean-squared error 1/(2B) sum (out - T)^2 and its exact gradients by
    backpropagation (reverse-mode chain rule, layer by layer)."""
    B = X.shape[1]
    out, (zs, hs) = mlp_forward(Ws, bs, X)
    diff = out - T
    loss = 0.5 * float(np.sum(diff * diff)) / B
    g = diff / B
    gW, gb = [None] * len(Ws), [None] * len(Ws)
    for li in range(len(Ws) - 1, -1, -1):
        if li < len(Ws) - 1:
            g = g * dsilu(zs[li])
        gW[li] = g @ hs[li].T
        gb[li] = g.sum(axis=1)
        g = Ws[li].T @ g
    return loss, gW, gb


def simplex_project(y):
    """Euclidean projection of each column of y onto {x >= 0, sum x = 1}:
    sort descending, find the largest rho with u_rho > (sum_{j<=rho} u_j - 1)
    / rho, shift by theta = (sum_{j<=rho} u_j - 1)/rho and clip at zero
    (Held, Wolfe and Crowder 1974; stated this way by Duchi et al. 2008)."""
    y = np.asarray(y, dtype=np.float64)
    col = y.ndim == 1
    Y = y.reshape(y.shape[0], -1)
    out = np.empty_like(Y)
    for c in range(Y.shape[1]):
        u = np.sort(Y[:, c])[::-1]
        css = np.cumsum(u)
        rho = 0
        for j in range(u.size):
            if u[j] - (css[j] - 1.0) / (j + 1) > 0:
                rho = j + 1
        theta = (css[rho - 1] - 1.0) / rho
        out[:, c] = np.maximum(Y[:, c] - theta, 0.0)
    return out[:, 0] if col else out


def surrogate_step(Ws, bs, v, dt, x, params=None, net=None):
    """Projected surrogate prediction of the implicit Euler step, (9, batch).

    Scaled form (kinetic parameter block `params` given): with
    z = dt A(v) x and s = ||z||_1 the network sees (v_n, dt_n, z/s) and its
    output y gives the increment s*y; the exact increment is J^-1 z with
    ||J^-1||_1 = 1, so the target J^-1 z / s is a smooth function of the
    inputs.  Raw form (params None): the network sees (v_n, dt_n, x) and its
    output is the increment itself.

    net: the network as a function of the (11, batch) inputs; by default the
    MLP (Ws, bs).  Tests put known functions there (zero, identity on the
    state inputs, the exact target) to check the composition around it."""
    if net is None:
        def net(X):
            return mlp_forward(Ws, bs, X)[0]
    x = np.asarray(x, dtype=np.float64).reshape(9, -1)
    v = np.atleast_1d(np.asarray(v, dtype=np.float64))
    if params is None:
        return simplex_project(x + net(surrogate_inputs(v, dt, x)))
    z = np.stack([dt * (kin9_matrix(params, v[c]) @ x[:, c]) for c in range(x.shape[1])],
                 axis=1)
    s = np.sum(np.abs(z), axis=0)
    zn = np.where(s > 0, z / np.where(s > 0, s, 1.0), 0.0)
    out = net(surrogate_inputs(v, dt, zn))
    return simplex_project(x + out * s[None, :])


def kin9_residual(params, v, dt, x_old, y):
    """F(y) = y - x - dt A(v) y per column (the implicit Euler residual)."""
    v = np.atleast_1d(v)
    R = np.empty_like(np.asarray(y, dtype=np.float64))
    for c in range(v.size):
        A = kin9_matrix(params, v[c])
        R[:, c] = y[:, c] - x_old[:, c] - dt * (A @ y[:, c])
    return R


class pade_mode:
    """Context manager: cnexp with the (1,1) Pade approximant of exp(-x)
    (Section 5.2) inside the block."""

    def __enter__(self):
        ctypes.c_int.in_dll(lib(), "orc_pade_mode").value = 1
        return self

    def __exit__(self, *exc):
        ctypes.c_int.in_dll(lib(), "orc_pade_mode").value = 0
        return False


def cnexp_factor(x: float) -> float:
    return lib().orc_cnexp_factor(float(x))


def step_cable(mechs, states, v, n_nodes, parent, ga, gb, dt, cm=1.0, nsteps=1,
               tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    """nsteps cable steps (orc_step_cable); returns (v, rhs, d, states) with
    rhs/d the last step's assembled values (before the solve)."""
    keep = []
    arr = (_OrcMech * len(mechs))()
    out_states = []
    for k, m in enumerate(mechs):
        p, ni = _f64(m["params"]), _i32(m["node_index"])
        s = _f64(states[k]).copy()
        keep += [p, ni]
        out_states.append(s)
        arr[k].type = int(m["type"])
        arr[k].n = ni.size
        arr[k].node_index = ni.ctypes.data
        arr[k].params = p.ctypes.data
        arr[k].states = s.ctypes.data
    vv = _f64(v).copy()
    rhs, d = np.zeros(n_nodes), np.zeros(n_nodes)
    par, a, b = _i32(parent), _f64(ga), _f64(gb)
    lib().orc_step_cable(len(mechs), ctypes.cast(arr, ctypes.c_void_p), int(n_nodes),
                         _p(par), _p(a), _p(b), float(dt), float(cm), _p(vv), _p(rhs),
                         _p(d), int(nsteps), float(tol), int(max_iter))
    return vv, rhs, d, out_states


def step_ions(mechs, states, v, n_nodes, dt, cm=1.0, nsteps=1, clamp_v=False,
              tol=NEWTON_TOL, max_iter=NEWTON_MAX_ITER):
    """nsteps steps with per-node ion currents (orc_step_ions); mechs may
    carry an "ion" tag.  Returns (v, rhs, d, ion [4][n_nodes], states) after
    the last step (ion row 0 unused)."""
    keep = []
    arr = (_OrcMech * len(mechs))()
    out_states = []
    for k, m in enumerate(mechs):
        p, ni = _f64(m["params"]), _i32(m["node_index"])
        s = _f64(states[k]).copy()
        keep += [p, ni]
        out_states.append(s)
        arr[k].type = int(m["type"])
        arr[k].ion = int(m.get("ion", ION_NONE))
        arr[k].n = ni.size
        arr[k].node_index = ni.ctypes.data
        arr[k].params = p.ctypes.data
        arr[k].states = s.ctypes.data
    vv = _f64(v).copy()
    rhs, d = np.zeros(n_nodes), np.zeros(n_nodes)
    ion = np.zeros((4, int(n_nodes)))
    ptrs = (ctypes.c_void_p * 4)(None, *[ion[k].ctypes.data for k in (1, 2, 3)])
    lib().orc_step_ions(len(mechs), ctypes.cast(arr, ctypes.c_void_p), int(n_nodes),
                        float(dt), float(cm), _p(vv), _p(rhs), _p(d),
                        ctypes.cast(ptrs, ctypes.c_void_p), int(nsteps),
                        int(bool(clamp_v)), float(tol), int(max_iter))
    return vv, rhs, d, ion, out_states
