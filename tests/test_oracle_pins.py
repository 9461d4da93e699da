"""Pins of the FP64 CPU oracle against things other than itself.

Each test ties one oracle routine to a closed form, an invariant, a textbook
value, an independent algorithm (bisection, least squares, numpy's LAPACK
solve, RK4 at a tiny step, mpmath at 50 digits, finite differences) so that
a dropped term, a wrong sign, a wrong index or a transposed operand in the
oracle fails at least one of them:

  P1  cnexp closed form at clamped v                 test_p1_*
  P2  steady states (gates -> minf, kinetic -> null vector by lstsq)
  P3  HH resting potential by bisection of the steady-state current
  P4  kinetic conservation and positivity
  P5  RK4 brute force, first-order convergence of the step schemes
  P6  kinetic step == dense solve; 2-state closed form; Newton count
  P7  rate shapes at 50 digits; textbook HH values; vtrap limits
  P8  J^-1 >= 0 with unit column sums (the fallback error bound)
  P9  MLP gradients vs central differences; simplex projection vs bisection
  P10 accumulation vs brute-force per-node sums
  P11 analytic conductance vs central difference of the current
"""
import os

import mpmath
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W

HERE = os.path.dirname(os.path.abspath(__file__))


def golden(name):
    vals = {}
    with open(os.path.join(HERE, "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, v, tol = line.split()
            vals[k] = (float(v), float(tol))
    return vals


HH = W.hh_params()


def cortical_blocks():
    return W.cortical_type_params(2)


# ------------------------------------------------------------------- P7

mpmath.mp.dps = 50


def mp_rate(form, A, vh, k, v):
    u = (mpmath.mpf(v) - mpmath.mpf(vh)) / mpmath.mpf(k)
    A = mpmath.mpf(A)
    if form == 0:
        return A * mpmath.exp(u)
    if form == 1:
        return A / (1 + mpmath.exp(-u))
    if u == 0:
        return A
    return A * u / (1 - mpmath.exp(-u))


def test_p7_rate_shapes_vs_mpmath(orc):
    rng = np.random.default_rng(7)
    worst = 0.0
    for form in (0, 1, 2):
        for _ in range(300):
            A = 10 ** rng.uniform(-2, 0)
            vh = rng.uniform(-70, -20)
            k = rng.uniform(5, 30) * rng.choice([-1, 1])
            v = rng.uniform(-100, 60)
            ref = float(mp_rate(form, A, vh, k, v))
            got = orc.rate(form, A, vh, k, v)
            worst = max(worst, abs(got - ref) / abs(ref))
    assert worst < 4e-15, worst


def test_p7_linoid_near_zero_and_continuity(orc):
    # u within and just outside the Taylor branch, vs 50-digit evaluation
    for u in (0.0, 1e-12, -3e-9, 9.99e-7, -9.99e-7, 1.001e-6, -1.001e-6, 1e-4):
        v = -40.0 + 10.0 * u
        ref = float(mp_rate(2, 1.0, -40.0, 10.0, v))
        got = orc.rate(2, 1.0, -40.0, 10.0, v)
        assert abs(got - ref) <= 2e-15 * ref, (u, got, ref)


def test_p7_vtrap_limit_and_expm1_form(orc):
    g = golden("hh_rest_textbook.txt")
    # alpha_m(-40) = 0.1 vtrap(0, 10) = 1 exactly in the limit
    v, tol = g["alpha_m_at_-40"]
    assert abs(0.1 * orc.vtrap(0.0, 10.0) - v) <= tol
    v, tol = g["alpha_n_at_-55"]
    assert abs(0.01 * orc.vtrap(0.0, 10.0) - v) <= tol
    for x in (1e-3, -2.5, 7.0, 25.0, -30.0, 3e-7):
        ref = mpmath.mpf(x) / (mpmath.exp(mpmath.mpf(x) / 10) - 1)
        assert abs(orc.vtrap(x, 10.0) - float(ref)) <= 2e-15 * abs(float(ref))


def test_p7_hh_textbook_values(orc):
    g = golden("hh_rest_textbook.txt")
    minf, mtau = orc.hh_rates(HH, -65.0)
    for k, name in enumerate(("m_inf", "h_inf", "n_inf")):
        val, tol = g[name]
        assert abs(minf[k] - val) <= tol, (name, minf[k])
    # mtau = 1/(alpha+beta) at q10 = 1 (celsius 6.3): independent 50-digit
    v = mpmath.mpf(-65)
    am = 0.1 * (v + 40) / (1 - mpmath.exp(-(v + 40) / 10))
    bm = 4 * mpmath.exp(-(v + 65) / 18)
    assert abs(mtau[0] - float(1 / (am + bm))) < 1e-15 * mtau[0]


def test_p7_hh_temperature_factor(orc):
    p = HH.copy()
    p[6] = 16.3  # q10 = 3 -> mtau divides by exactly 3
    _, t1 = orc.hh_rates(HH, -50.0)
    _, t3 = orc.hh_rates(p, -50.0)
    np.testing.assert_allclose(t1 / t3, 3.0, rtol=1e-14)


def test_p7_generic_block_reproduces_hh(orc):
    # The HH gates written as generic cnexp gates (u-form constants derived
    # by hand: alpha_m = 0.1 vtrap(-(v+40),10) = 1.0 * u/(1-exp(-u)),
    # u = (v+40)/10, etc.) must agree with the textbook HH routine.
    gates = [
        (3, (2, 1.0, -40.0, 10.0), (0, 4.0, -65.0, -18.0)),
        (1, (0, 0.07, -65.0, -20.0), (1, 1.0, -35.0, 10.0)),
        (4, (2, 0.1, -55.0, 10.0), (0, 0.125, -65.0, -80.0)),
    ]
    p = W.cnexp_params(0.12, 50.0, gates, q10=3.0, celsius=6.3, t0=6.3)
    for v in np.linspace(-100, 60, 37):
        mi, mt = orc.hh_rates(HH, v)
        for gidx in range(3):
            a, b = orc.cnexp_rates(p, gidx, v)
            assert abs(a - mi[gidx]) <= 1e-14 * max(mi[gidx], 1e-300) + 1e-300
            assert abs(b - mt[gidx]) <= 1e-14 * mt[gidx]


# ------------------------------------------------------------------- P1

@pytest.mark.parametrize("which", ["hh", "cnexp"])
def test_p1_cnexp_closed_form(orc, which):
    n = 64
    v = np.linspace(-95.0, 45.0, n)
    ni = np.arange(n, dtype=np.int32)
    if which == "hh":
        mtype, p = W.TYPE_HH, HH
    else:
        mtype, p = W.TYPE_CNEXP, cortical_blocks()[0]
    ng = orc.n_states(mtype, p)
    rng = np.random.default_rng(1)
    s0 = rng.uniform(0, 1, size=(ng, n))
    dt, N = 0.025, 57
    s = s0.copy()
    for _ in range(N):
        s = orc.mech_state(mtype, p, ni, v, s, dt)
    for i in range(n):
        for g in range(ng):
            if which == "hh":
                mi, mt = orc.hh_rates(p, v[i])
                minf, mtau = mi[g], mt[g]
            else:
                minf, mtau = orc.cnexp_rates(p, g, v[i])
            exact = minf + (s0[g, i] - minf) * np.exp(-N * dt / mtau)
            assert abs(s[g, i] - exact) <= 1e-13 * max(abs(exact), 1e-3), \
                (g, i, s[g, i], exact)


# ------------------------------------------------------------------- P2

def test_p2_gates_converge_to_minf(orc):
    p = cortical_blocks()[2]
    n = 16
    v = np.linspace(-80, 30, n)
    ni = np.arange(n, dtype=np.int32)
    s = np.zeros((3, n))
    for _ in range(400):
        s = orc.mech_state(W.TYPE_CNEXP, p, ni, v, s, 0.5)
    init = orc.mech_init(W.TYPE_CNEXP, p, ni, v)
    for i in range(n):
        for g in range(3):
            minf, mtau = orc.cnexp_rates(p, g, v[i])
            if 400 * 0.5 / mtau > 60:  # converged to within exp(-60)
                assert abs(s[g, i] - minf) < 1e-13
            assert init[g, i] == minf


def test_p2_kinetic_stationary_vs_lstsq(orc):
    p = W.kin9_params(W.Stream(4, 401))
    for v in np.linspace(-100, 60, 17):
        A = orc.kin9_matrix(p, v)
        pi = orc.kin9_stationary(p, v)
        M = np.vstack([A, np.ones((1, 9))])
        rhs = np.zeros(10)
        rhs[-1] = 1
        ref = np.linalg.lstsq(M, rhs, rcond=None)[0]
        np.testing.assert_allclose(pi, ref, rtol=1e-10, atol=1e-14)
        assert np.all(pi > 0)
        # the stationary distribution is a fixed point of the step
        y, it, sw = orc.kin9_newton(A, 0.025, pi)
        np.testing.assert_allclose(y, pi, rtol=1e-12, atol=1e-15)


def test_p2_kinetic_relaxes_to_stationary(orc):
    p = W.kin9_params(W.Stream(4, 401))
    n = 8
    v = np.linspace(-90, 50, n)
    ni = np.arange(n, dtype=np.int32)
    x = W.Stream(9, 1).dirichlet(n, 9)
    for _ in range(60):
        x = orc.mech_state(W.TYPE_KIN9, p, ni, v, x, 50.0)
    for i in range(n):
        np.testing.assert_allclose(x[:, i], orc.kin9_stationary(p, v[i]),
                                   rtol=1e-9, atol=1e-12)


def test_p2_kinetic_matrix_structure(orc):
    p = W.kin9_params(W.Stream(4, 401))
    A = orc.kin9_matrix(p, -20.0)
    np.testing.assert_allclose(A.sum(axis=0), 0.0, atol=1e-12)
    off = A - np.diag(np.diag(A))
    assert np.all(off >= 0)
    # nonzero pattern: lattice neighbours only
    for i in range(9):
        for j in range(9):
            if i == j:
                continue
            ai, bi, aj, bj = i // 3, i % 3, j // 3, j % 3
            nb = abs(ai - aj) + abs(bi - bj) == 1
            assert (off[i, j] > 0) == nb
    # a single edge's forward rate, from the parameter block by hand
    af, bf = p[3], p[4]  # edge 0: state 0 -> state 1
    assert abs(A[1, 0] - af * np.exp(bf * -20.0)) < 1e-15 * A[1, 0]
    ab, bb = p[5], p[6]  # state 1 -> state 0
    assert abs(A[0, 1] - ab * np.exp(-bb * -20.0)) < 1e-15 * A[0, 1]


# ------------------------------------------------------------------- P3

def test_p3_hh_rest_potential(orc):
    g = golden("hh_rest_textbook.txt")
    ni = np.zeros(1, dtype=np.int32)

    def iss(v):
        # steady-state HH current through the oracle's gates and current
        s = orc.mech_init(W.TYPE_HH, HH, ni, np.array([v]))
        c, _ = orc.mech_currents(W.TYPE_HH, HH, ni, np.array([v]), s)
        return c[0]

    lo, hi = -80.0, -50.0
    assert iss(lo) < 0 < iss(hi)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if iss(mid) < 0:
            lo = mid
        else:
            hi = mid
    vrest = 0.5 * (lo + hi)
    val, tol = g["v_rest_mV"]
    assert abs(vrest - val) < tol, vrest
    # an unstimulated compartment started near rest settles there
    mech = dict(type=W.TYPE_HH, params=HH, node_index=ni)
    for v0 in (-70.0, -67.0, -62.0):
        s0 = orc.mech_init(W.TYPE_HH, HH, ni, np.array([v0]))
        v, rhs, d, _ = orc.step([mech], [s0], np.array([v0]), 1, 0.025,
                                nsteps=20000)
        assert abs(v[0] - vrest) < 1e-6, (v0, v[0], vrest)


# ------------------------------------------------------------------- P4

def test_p4_kinetic_conservation_positivity(orc):
    d = W.kin9_clamped(256, seed=4)
    m = d["mechs"][0]
    x = d["x0"].copy()
    N = 200
    for _ in range(N):
        x = orc.mech_state(m["type"], m["params"], m["node_index"], d["v0"],
                           x, 0.025)
    assert np.max(np.abs(x.sum(axis=0) - 1.0)) <= 1e-14 * N
    assert np.all(x >= 0.0)


# ------------------------------------------------------------------- P5

def _rk4(f, y, h, n):
    for _ in range(n):
        k1 = f(y)
        k2 = f(y + 0.5 * h * k1)
        k3 = f(y + 0.5 * h * k2)
        k4 = f(y + h * k3)
        y = y + h / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return y


def test_p5_kinetic_rk4_first_order(orc):
    p = W.kin9_params(W.Stream(4, 401))
    v = np.array([-30.0, 10.0])
    ni = np.arange(2, dtype=np.int32)
    x0 = W.Stream(11, 1).dirichlet(2, 9)
    T = 0.4
    ref = np.stack([_rk4(lambda y, A=orc.kin9_matrix(p, v[i]): A @ y,
                         x0[:, i], 1e-4, int(round(T / 1e-4)))
                    for i in range(2)], axis=1)
    errs = []
    for dt in (0.025, 0.0125, 0.00625):
        x = x0.copy()
        for _ in range(int(round(T / dt))):
            x = orc.mech_state(W.TYPE_KIN9, p, ni, v, x, dt)
        errs.append(np.max(np.abs(x - ref)))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.7 < r1 < 2.3 and 1.8 < r2 < 2.2, errs


def test_p5_hh_rk4_convergence(orc):
    """Full HH ODE (v and gates) by RK4 at 1e-4 ms vs the staggered scheme.

    cm dv/dt = -I (units: dv/dt [mV/ms] = -1000 I [mA/cm2] / cm [uF/cm2]);
    dx/dt = (xinf - x)/xtau for x in m, h, n.  The scheme's error must fall
    at first order; the measured orders are recorded in the design notes.
    """
    ni = np.zeros(1, dtype=np.int32)
    mech = dict(type=W.TYPE_HH, params=HH, node_index=ni)

    def f(y):
        v = y[0]
        mi, mt = orc.hh_rates(HH, v)
        s = y[1:].reshape(3, 1)
        c, _ = orc.mech_currents(W.TYPE_HH, HH, ni, np.array([v]), s)
        return np.concatenate([[-1000.0 * c[0]], (mi - y[1:]) / mt])

    v0 = -58.0
    s0 = orc.mech_init(W.TYPE_HH, HH, ni, np.array([-65.0]))
    T = 2.0
    ref = _rk4(f, np.concatenate([[v0], s0[:, 0]]), 1e-4, int(round(T / 1e-4)))
    errs = []
    for dt in (0.025, 0.0125, 0.00625):
        v, _, _, st = orc.step([mech], [s0], np.array([v0]), 1, dt,
                               nsteps=int(round(T / dt)))
        errs.append(abs(v[0] - ref[0]))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 1.6 < r1 < 2.4 and 1.7 < r2 < 2.3, errs


# ------------------------------------------------------------------- P6

def test_p6_kinetic_step_is_dense_solve(orc):
    p = W.kin9_params(W.Stream(4, 401))
    rng = np.random.default_rng(3)
    for v in (-100.0, -37.0, 0.0, 60.0):
        A = orc.kin9_matrix(p, v)
        x = W.Stream(int(v + 1000), 2).dirichlet(1, 9)[:, 0]
        for dt in (0.025, 0.3):
            y, it, sw = orc.kin9_newton(A, dt, x)
            ref = np.linalg.solve(np.eye(9) - dt * A, x)
            np.testing.assert_allclose(y, ref, rtol=1e-12, atol=1e-15)
            assert it <= 2  # linear: one update, then a negligible second
            assert sw == 0  # column diagonally dominant M-matrix: no swaps
    _ = rng


def test_p6_two_state_closed_form(orc):
    a, b, dt = 2.5, 0.7, 0.1
    A = np.zeros((9, 9))
    A[1, 0], A[0, 0] = a, -a   # 0 -> 1 at rate a
    A[0, 1], A[1, 1] = b, -b   # 1 -> 0 at rate b
    x = np.zeros(9)
    x[0], x[1] = 0.3, 0.7
    y, it, sw = orc.kin9_newton(A, dt, x)
    s = x[0] + x[1]
    y1 = (x[1] + dt * a * s) / (1 + dt * (a + b))
    assert abs(y[1] - y1) < 1e-15 and abs(y[0] - (s - y1)) < 1e-15
    assert np.all(y[2:] == x[2:])


def test_lu_solve_of_any_size_vs_numpy(orc):
    """The dense LU with partial pivoting and its solve on systems larger
    than any fixed buffer (the cable form's cells reach 400 nodes)."""
    rng = np.random.default_rng(12)
    for n in (1, 9, 65, 200, 401):
        M = rng.normal(size=(n, n)) + n * np.eye(n)
        b = rng.normal(size=n)
        LU, perm, _ = orc.lu_pp(M)
        x = orc.lu_solve(LU, perm, b)
        np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)


def test_p6_lu_pp_vs_numpy(orc):
    rng = np.random.default_rng(5)
    for _ in range(20):
        M = rng.normal(size=(9, 9))
        LU, perm, sw = orc.lu_pp(M)
        b = rng.normal(size=9)
        np.testing.assert_allclose(orc.lu_solve(LU, perm, b),
                                   np.linalg.solve(M, b), rtol=1e-10, atol=1e-12)


# ------------------------------------------------------------------- P8

def test_p8_inverse_is_column_stochastic(orc):
    p = W.kin9_params(W.Stream(4, 401))
    for v in np.linspace(-100, 60, 9):
        A = orc.kin9_matrix(p, v)
        Jinv = np.linalg.inv(np.eye(9) - 0.025 * A)
        assert np.all(Jinv >= -1e-15)
        np.testing.assert_allclose(Jinv.sum(axis=0), 1.0, rtol=1e-13)
        # residual bound: ||y - y*||_1 <= ||F(y)||_1 for any y
        x = W.Stream(int(v + 500), 3).dirichlet(1, 9)[:, 0]
        ystar, _, _ = orc.kin9_newton(A, 0.025, x)
        y = ystar + 1e-3 * np.sin(np.arange(9) + v)
        F = y - x - 0.025 * A @ y
        assert np.sum(np.abs(y - ystar)) <= np.sum(np.abs(F)) * (1 + 1e-12)


# ------------------------------------------------------------------- P9

def test_p9_mlp_gradients_vs_central_differences(orc):
    Ws, bs = W.mlp_init(3, widths=(11, 6, 5, 4, 9), out_scale=1.0)
    v, dt, x, _ = W.surrogate_samples(5, seed=8)
    X = orc.surrogate_inputs(v, dt, x)
    T = np.sin(np.arange(45)).reshape(9, 5) * 0.1
    loss, gW, gb = orc.mlp_loss_grad(Ws, bs, X, T)
    h = 1e-6
    for li in range(4):
        for idx in [(0, 0), (1, 2), (Ws[li].shape[0] - 1, Ws[li].shape[1] - 1)]:
            Wp = [w.copy() for w in Ws]
            Wm = [w.copy() for w in Ws]
            Wp[li][idx] += h
            Wm[li][idx] -= h
            lp, _, _ = orc.mlp_loss_grad(Wp, bs, X, T)
            lm, _, _ = orc.mlp_loss_grad(Wm, bs, X, T)
            fd = (lp - lm) / (2 * h)
            assert abs(fd - gW[li][idx]) <= 1e-7 * max(abs(fd), 1e-3), (li, idx)
        bp = [b.copy() for b in bs]
        bm = [b.copy() for b in bs]
        bp[li][1] += h
        bm[li][1] -= h
        fd = (orc.mlp_loss_grad(Ws, bp, X, T)[0]
              - orc.mlp_loss_grad(Ws, bm, X, T)[0]) / (2 * h)
        assert abs(fd - gb[li][1]) <= 1e-7 * max(abs(fd), 1e-3)


def _project_bisect(y):
    lo, hi = np.min(y) - 1.0, np.max(y)
    for _ in range(200):
        th = 0.5 * (lo + hi)
        if np.sum(np.maximum(y - th, 0)) > 1:
            lo = th
        else:
            hi = th
    return np.maximum(y - 0.5 * (lo + hi), 0)


def test_p9_simplex_projection(orc):
    rng = np.random.default_rng(11)
    for _ in range(200):
        y = rng.normal(size=9) * rng.choice([0.01, 0.3, 3.0])
        x = orc.simplex_project(y)
        assert abs(x.sum() - 1) < 1e-14 and np.all(x >= 0)
        np.testing.assert_allclose(x, _project_bisect(y), atol=1e-12)
    # points already on the simplex are fixed
    z = W.Stream(1, 1).dirichlet(10, 9)
    np.testing.assert_allclose(orc.simplex_project(z), z, atol=1e-15)
    # a vertex-dominated point goes to the vertex
    e = np.zeros(9)
    e[4] = 5.0
    np.testing.assert_allclose(orc.simplex_project(e), np.eye(9)[4])


# ------------------------------------------- P9b: the surrogate composition
# oracle.surrogate_step wraps the network: z = dt A(v) x, s = ||z||_1, the
# network sees (v_n, dt_n, z/s), the increment is s * output, and the sum is
# projected onto the simplex.  Known functions in place of the network pin
# every piece of that wrapper against the implicit-Euler step (Section 5.2)
# and the explicit one, independently of any trained weights.

def _implicit_euler_dense(A, dt, x):
    return np.linalg.solve(np.eye(9) - dt * A, x)


def test_p9b_surrogate_inputs_normalisation(orc):
    # the training ranges v in [-100, 60] mV and dt in [0.0125, 0.05] ms map
    # onto [-1, 1]; their midpoints onto 0; the state rows pass unchanged
    X = orc.surrogate_inputs([-100.0, 60.0, -20.0], [0.0125, 0.05, 0.03125],
                             np.arange(27.0).reshape(9, 3))
    assert X.shape == (11, 3)
    np.testing.assert_allclose(X[0], [-1.0, 1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(X[1], [-1.0, 1.0, 0.0], atol=1e-14)
    np.testing.assert_array_equal(X[2:], np.arange(27.0).reshape(9, 3))


def test_p9b_exact_network_gives_the_implicit_euler_step(orc):
    """With the network replaced by the exact map z/s -> J^-1 z/s, the
    wrapped prediction is the dense implicit-Euler step to rounding; the
    network's state inputs are the direction of dt A x, with unit 1-norm and
    zero sum (the columns of A sum to zero)."""
    p = W.kin9_params(W.Stream(4, 401))
    v = np.array([-100.0, -63.0, -20.5, 0.0, 37.0, 60.0])
    dts = np.array([0.0125, 0.025, 0.05, 0.025, 0.03, 0.025])
    x = W.Stream(9, 2).dirichlet(v.size, 9)
    x[:, 3] = orc.kin9_stationary(p, v[3])          # s ~ 0: the stationary point
    for dt in (0.0125, 0.025, 0.05):
        def exact(X, dt=dt):
            zn = X[2:]
            col_l1 = np.sum(np.abs(zn), axis=0)
            assert np.all((np.abs(col_l1 - 1) < 1e-14) | (col_l1 == 0)), col_l1
            # zero sum up to rounding; at the stationary point (column 3) z is
            # rounding noise and its direction is arbitrary
            assert np.all(np.delete(np.abs(zn.sum(axis=0)), 3) < 1e-14)
            return np.stack([np.linalg.solve(np.eye(9) - dt * orc.kin9_matrix(p, v[c]), zn[:, c])
                             for c in range(v.size)], axis=1)
        got = orc.surrogate_step(None, None, v, dt, x, params=p, net=exact)
        for c in range(v.size):
            want = _implicit_euler_dense(orc.kin9_matrix(p, v[c]), dt, x[:, c])
            np.testing.assert_allclose(got[:, c], want, rtol=0, atol=1e-14)
    # dt = 0: z = 0 exactly, s = 0, and the step returns x itself
    got = orc.surrogate_step(None, None, v, 0.0, x, params=p, net=lambda X: np.ones((9, v.size)))
    np.testing.assert_allclose(got, x, atol=1e-15)


def test_p9b_identity_network_gives_the_explicit_euler_step(orc):
    """A one-layer network that copies its state inputs makes the increment
    s * z/s = dt A x, so the prediction is the projected explicit Euler step
    x + dt A x (on the simplex already for small dt: A's off-diagonals are
    nonnegative and its columns sum to zero)."""
    p = W.kin9_params(W.Stream(4, 401))
    v = np.array([-80.0, -10.0, 45.0])
    x = W.Stream(9, 5).dirichlet(3, 9)
    Wid = np.hstack([np.zeros((9, 2)), np.eye(9)])
    dt = 1e-3
    got = orc.surrogate_step([Wid], [np.zeros(9)], v, dt, x, params=p)
    for c in range(3):
        A = orc.kin9_matrix(p, v[c])
        want = x[:, c] + dt * A @ x[:, c]
        assert np.all(want >= 0)
        np.testing.assert_allclose(got[:, c], want, rtol=0, atol=1e-15)
    # the raw form with a zero network returns the projected input
    Z = [np.zeros((9, 11))]
    np.testing.assert_allclose(orc.surrogate_step(Z, [np.zeros(9)], v, 0.025, x), x,
                               atol=1e-15)


def test_p9b_mlp_forward_closed_form(orc):
    # two layers, one unit each: out = 2 silu(z) + 1 with silu(1) = e/(e + 1)
    # and silu(-2) = -2/(1 + e^2); SiLU on the hidden layer only
    X = np.array([[1.0, -2.0]])
    out, _ = orc.mlp_forward([np.array([[1.0]]), np.array([[2.0]])],
                             [np.zeros(1), np.ones(1)], X)
    e = np.e
    np.testing.assert_allclose(out[0], [2 * e / (e + 1) + 1, 2 * (-2 / (1 + e * e)) + 1],
                               rtol=1e-15)


# ------------------------------------------------------------------ P10

def test_p10_accumulation_vs_brute_force(orc):
    d = W.cortical_mix(300, seed=5)
    rng = np.random.default_rng(2)
    rhs0 = rng.normal(size=300)
    d0 = rng.uniform(0.1, 1, size=300)
    for m in d["mechs"]:
        ng = orc.n_states(m["type"], m["params"])
        s = rng.uniform(0, 1, size=(ng, m["node_index"].size))
        rhs, dd = orc.mech_cur(m["type"], m["params"], m["node_index"], d["v0"],
                               s, rhs0, d0)
        c, g = orc.mech_currents(m["type"], m["params"], m["node_index"],
                                 d["v0"], s)
        bf_r, bf_d = rhs0.copy(), d0.copy()
        per_node = {}
        for j, node in enumerate(m["node_index"]):
            per_node.setdefault(int(node), []).append(j)
        for node, js in per_node.items():
            bf_r[node] -= sum(c[j] for j in js)
            bf_d[node] += sum(g[j] for j in js)
        np.testing.assert_allclose(rhs, bf_r, rtol=1e-13, atol=1e-15)
        np.testing.assert_allclose(dd, bf_d, rtol=1e-13, atol=1e-15)
        # and a generic current from its definition g = gbar prod x^p
        p = m["params"]
        j = min(5, m["node_index"].size - 1)
        gg = p[1]
        for k in range(int(p[0])):
            gg *= s[k, j] ** int(p[6 + 9 * k])
        assert abs(g[j] - gg) <= 1e-14 * gg + 1e-300
        assert abs(c[j] - gg * (d["v0"][m["node_index"][j]] - p[2])) <= \
            1e-13 * abs(c[j]) + 1e-300


# ------------------------------------------------------------------ P11

@pytest.mark.parametrize("which", ["hh", "cnexp", "kin9"])
def test_p11_conductance_is_dIdv(orc, which):
    n = 32
    ni = np.arange(n, dtype=np.int32)
    v = np.linspace(-90, 40, n)
    rng = np.random.default_rng(4)
    if which == "hh":
        mt, p = W.TYPE_HH, HH
    elif which == "cnexp":
        mt, p = W.TYPE_CNEXP, cortical_blocks()[0]
    else:
        mt, p = W.TYPE_KIN9, W.kin9_params(W.Stream(4, 401))
    s = rng.uniform(0, 1, size=(orc.n_states(mt, p), n))
    h = 1e-4
    _, g = orc.mech_currents(mt, p, ni, v, s)
    cp, _ = orc.mech_currents(mt, p, ni, v + h, s)
    cm, _ = orc.mech_currents(mt, p, ni, v - h, s)
    np.testing.assert_allclose(g, (cp - cm) / (2 * h), rtol=1e-7, atol=1e-12)


# ------------------------------------------------------------- step order

def test_step_matches_hand_composition(orc):
    """One network step equals zero -> cur (list order) -> d += cm/dt*1e-3
    -> v += rhs/d -> state, composed here from the per-mechanism routines."""
    d = W.cortical_mix(200, seed=7)
    mechs = d["mechs"]
    states = [orc.mech_init(m["type"], m["params"], m["node_index"], d["v0"])
              for m in mechs]
    dt, cm = 0.025, 1.0
    v1, rhs1, d1, st1 = orc.step(mechs, states, d["v0"], 200, dt, cm)
    rhs, dd = np.zeros(200), np.zeros(200)
    for m, s in zip(mechs, states):
        rhs, dd = orc.mech_cur(m["type"], m["params"], m["node_index"],
                               d["v0"], s, rhs, dd)
    dd = dd + 1e-3 * cm / dt
    v = d["v0"] + rhs / dd
    np.testing.assert_array_equal(rhs1, rhs)
    np.testing.assert_array_equal(d1, dd)
    np.testing.assert_array_equal(v1, v)
    for m, s, s1 in zip(mechs, states, st1):
        np.testing.assert_array_equal(
            s1, orc.mech_state(m["type"], m["params"], m["node_index"], v, s, dt))


def test_kin9_current_reads_open_state(orc):
    """g = gbar * x_open with the open state (2, 0) = index 6 of the lattice."""
    p = W.kin9_params(W.Stream(4, 401))
    ni = np.arange(9, dtype=np.int32)
    v = np.full(9, -20.0)
    s = np.eye(9)  # instance k sits entirely in state k
    c, g = orc.mech_currents(W.TYPE_KIN9, p, ni, v, s)
    expect = np.zeros(9)
    expect[W.KIN9_OPEN] = p[0]
    np.testing.assert_array_equal(g, expect)
    assert c[W.KIN9_OPEN] == p[0] * (-20.0 - p[1])


def test_step_clamped_voltage(orc):
    d = W.kin9_clamped(16, seed=4)
    m = d["mechs"][0]
    v, rhs, dd, st = orc.step([m], [d["x0"]], d["v0"], 16, 0.025, nsteps=3,
                              clamp_v=True)
    np.testing.assert_array_equal(v, d["v0"])
    # rhs/d still hold the last step's accumulation
    x2 = d["x0"]
    for _ in range(2):
        x2 = orc.mech_state(m["type"], m["params"], m["node_index"], d["v0"],
                            x2, 0.025)
    r, g = orc.mech_cur(m["type"], m["params"], m["node_index"], d["v0"], x2,
                        np.zeros(16), np.zeros(16))
    np.testing.assert_array_equal(rhs, r)
    np.testing.assert_array_equal(dd, g + 1e-3 / 0.025)


def test_kin9_residual_vanishes_at_dense_solution(orc):
    p = W.kin9_params(W.Stream(4, 401))
    v = np.array([-80.0, -10.0, 45.0])
    x = W.Stream(5, 5).dirichlet(3, 9)
    y = np.stack([np.linalg.solve(np.eye(9) - 0.025 * orc.kin9_matrix(p, v[c]),
                                  x[:, c]) for c in range(3)], axis=1)
    assert np.max(np.abs(orc.kin9_residual(p, v, 0.025, x, y))) < 1e-15
    r = orc.kin9_residual(p, v, 0.025, x, x)   # y = x leaves -dt A x
    assert np.max(np.abs(r.sum(axis=0))) < 1e-15   # columns of A sum to 0
    assert np.max(np.abs(r)) > 1e-6


def test_pade_factor_and_second_order(orc):
    """(1,1) Pade cnexp: the factor is 2x/(2+x), it matches 1 - exp(-x) to
    x^3/12 + O(x^4), and the clamped-v gate converges at second order to the
    exact cnexp solution."""
    for x in (1e-3, 1e-2, 0.1, 0.5):
        with orc.pade_mode():
            f = orc.cnexp_factor(x)
        assert abs(f - 2 * x / (2 + x)) <= 2.5e-16 + 1e-15 * f  # 1 - R cancels
        assert abs(f - (1 - np.exp(-x))) <= x ** 3 / 12 * 1.2 + 1e-17
    assert orc.cnexp_factor(0.3) == 1 - np.exp(-0.3)      # default: exact
    p = cortical_blocks()[1]
    v = np.array([-30.0])
    ni = np.zeros(1, dtype=np.int32)
    minf, mtau = orc.cnexp_rates(p, 0, v[0])
    T, m0 = 2.0, np.array([[0.05]])
    exact = minf + (m0[0, 0] - minf) * np.exp(-T / mtau)
    errs = []
    for dt in (0.1, 0.05, 0.025):
        s = m0.copy()
        with orc.pade_mode():
            for _ in range(int(round(T / dt))):
                s = orc.mech_state(W.TYPE_CNEXP, p, ni, v, s, dt)
        errs.append(abs(s[0, 0] - exact))
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5, errs


def _cable_case(seed=3, n_cells=6, size_lo=4, size_hi=25):
    cab = W.cable_cells(n_cells, seed=seed, size_lo=size_lo, size_hi=size_hi)
    wl = W.cortical_mix(cab["n_nodes"], seed=seed + 10)
    return cab, wl


def test_cable_without_coupling_is_the_isolated_step(orc):
    cab, wl = _cable_case()
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
          for m in wl["mechs"]]
    z = np.zeros(cab["n_nodes"])
    a = orc.step_cable(wl["mechs"], st, wl["v0"], cab["n_nodes"], cab["parent"], z, z,
                       0.025, nsteps=3)
    b = orc.step(wl["mechs"], st, wl["v0"], cab["n_nodes"], 0.025, nsteps=3)
    np.testing.assert_allclose(a[0], b[0], rtol=1e-15, atol=1e-13)
    np.testing.assert_array_equal(a[2], b[2])


@pytest.mark.parametrize("n_cells,size_lo,size_hi", [(6, 4, 25), (3, 150, 400)])
def test_cable_step_solves_the_assembled_tree_system(orc, n_cells, size_lo, size_hi):
    """v_new - v = M^-1 rhs with M, rhs assembled here from the membrane
    terms (rhs0, d0 of the uncoupled step) and the axial conductances; small
    cells and cells of the benchmark's largest sizes (up to 400 nodes)."""
    cab, wl = _cable_case(seed=4, n_cells=n_cells, size_lo=size_lo, size_hi=size_hi)
    n = cab["n_nodes"]
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
          for m in wl["mechs"]]
    _, rhs0, d0, _ = orc.step(wl["mechs"], st, wl["v0"], n, 0.025, nsteps=1)
    v1, rhs1, d1, _ = orc.step_cable(wl["mechs"], st, wl["v0"], n, cab["parent"], cab["ga"],
                                     cab["gb"], 0.025, nsteps=1)
    M = np.diag(d0.copy())
    r = rhs0.copy()
    v0 = wl["v0"]
    for i in range(n):
        p = cab["parent"][i]
        if p < 0:
            continue
        M[i, i] += cab["ga"][i]
        M[p, p] += cab["gb"][i]
        M[i, p] -= cab["ga"][i]
        M[p, i] -= cab["gb"][i]
        r[i] += cab["ga"][i] * (v0[p] - v0[i])
        r[p] += cab["gb"][i] * (v0[i] - v0[p])
    np.testing.assert_allclose(v1 - v0, np.linalg.solve(M, r), rtol=1e-9, atol=1e-12)
    np.testing.assert_allclose(d1, np.diag(M), rtol=1e-14)
    np.testing.assert_allclose(rhs1, r, rtol=1e-12, atol=1e-14)


def test_cable_symmetric_twins_carry_no_axial_current(orc):
    """Two identical compartments coupled symmetrically, with the same state
    and voltage, evolve exactly like one uncoupled compartment."""
    ni = np.array([0, 1], dtype=np.int32)
    mech = dict(type=W.TYPE_HH, params=W.hh_params(), node_index=ni)
    v0 = np.array([-58.0, -58.0])
    s0 = orc.mech_init(W.TYPE_HH, W.hh_params(), ni, v0)
    parent = np.array([-1, 0], dtype=np.int32)
    g = np.array([0.0, 5.0])
    vc, _, _, sc = orc.step_cable([mech], [s0], v0, 2, parent, g, g, 0.025, nsteps=400)
    vs, _, _, ss = orc.step([mech], [s0], v0, 2, 0.025, nsteps=400)
    np.testing.assert_allclose(vc, vs, rtol=1e-12)
    assert vc[0] == vc[1]
