"""Pins of the oracle's small systems and ion currents.

  P12 3-state scheme: generator structure; detailed balance of the chain's
      stationary vector; one Newton update == numpy's dense solve; the
      2-state closed form; first-order convergence to scipy's expm.
  P13 calcium buffer: the rest state is a fixed point; closed forms with the
      buffer switched off and with binding switched off; total calcium
      conserved by binding; irreversible binding drains free calcium;
      quadratic Newton convergence (the exact Jacobian); fsolve agreement.
  P14 ion currents: HH splits into ina + ik + il with zeros at the reversal
      potentials; a tagged channel writes its per-node current sum; the
      whole calcium path (Ca channel -> ica -> buffer) against its closed
      form; ion recording leaves v, rhs and d untouched.
"""
import math

import numpy as np
import pytest
import scipy.linalg
import scipy.optimize

from paper_1905_02241_b300 import workloads as W


def kin3_rates(p, v):
    """(k_lo->hi, k_hi->lo) per edge, from the parameter layout."""
    return [(p[3 + 4 * e] * math.exp(p[4 + 4 * e] * v),
             p[5 + 4 * e] * math.exp(-p[6 + 4 * e] * v)) for e in range(3)]


# ------------------------------------------------------------------ P12

def test_p12_kin3_generator_structure(orc):
    p = W.kin3_params(W.Stream(12, 1))
    for v in (-90.0, -20.0, 35.0):
        A = orc.kin3_matrix(p, v)
        assert np.all(A - np.diag(np.diag(A)) >= 0)
        np.testing.assert_allclose(A.sum(axis=0), 0.0, atol=1e-15 * np.abs(A).max())
        r = kin3_rates(p, v)
        # (row = destination, column = source)
        assert A[1, 0] == pytest.approx(r[0][0], rel=1e-15)
        assert A[0, 1] == pytest.approx(r[0][1], rel=1e-15)
        assert A[2, 1] == pytest.approx(r[1][0], rel=1e-15)
        assert A[2, 0] == pytest.approx(r[2][0], rel=1e-15)
        assert A[0, 2] == pytest.approx(r[2][1], rel=1e-15)


def test_p12_kin3_chain_detailed_balance(orc):
    p = W.kin3_params(W.Stream(12, 2), chain=True)
    for v in (-80.0, -10.0, 40.0):
        pi = orc.kin_stationary_n(orc.kin3_matrix(p, v))
        r = kin3_rates(p, v)
        assert pi.sum() == pytest.approx(1.0, abs=1e-15)
        assert pi[1] / pi[0] == pytest.approx(r[0][0] / r[0][1], rel=1e-13)
        assert pi[2] / pi[1] == pytest.approx(r[1][0] / r[1][1], rel=1e-13)
    # INITIAL uses the same stationary vector
    ni = np.arange(3, dtype=np.int32)
    v = np.array([-80.0, -10.0, 40.0])
    s = orc.mech_init(W.TYPE_KIN3, p, ni, v)
    for i in range(3):
        np.testing.assert_allclose(orc.kin3_matrix(p, v[i]) @ s[:, i], 0.0, atol=1e-15)


def test_p12_kin3_step_is_one_dense_solve(orc):
    p = W.kin3_params(W.Stream(12, 3))
    for v in (-100.0, -40.0, 0.0, 60.0):
        A = orc.kin3_matrix(p, v)
        x = W.Stream(int(v + 300), 4).dirichlet(1, 3)[:, 0]
        for dt in (0.025, 0.5):
            y, it = orc.kin_newton_n(A, dt, x)
            ref = np.linalg.solve(np.eye(3) - dt * A, x)
            np.testing.assert_allclose(y, ref, rtol=1e-13, atol=1e-16)
            assert it <= 2
            y1, _ = orc.kin_newton_n(A, dt, x, max_iter=1)
            np.testing.assert_allclose(y1, y, rtol=0, atol=1e-15)  # rounding-size second update
            assert y.sum() == pytest.approx(x.sum(), abs=2e-16)
            assert np.all(y >= 0)


def test_p12_kin3_two_state_closed_form(orc):
    p = np.zeros(W.KIN3_NPARAM)
    p[0], p[1], p[2] = 0.1, -85.0, 1
    p[3:7] = (2.5, 0.0, 0.7, 0.0)  # edge (0,1): 0 -> 1 at 2.5, back at 0.7
    A = orc.kin3_matrix(p, -50.0)
    x = np.array([0.3, 0.7, 0.0])
    dt = 0.1
    y, _ = orc.kin_newton_n(A, dt, x)
    y1 = (x[1] + dt * 2.5 * 1.0) / (1 + dt * (2.5 + 0.7))
    assert abs(y[1] - y1) < 1e-15 and abs(y[0] - (1 - y1)) < 1e-15 and y[2] == 0.0


def test_p12_kin3_first_order_vs_expm(orc):
    p = W.kin3_params(W.Stream(12, 5))
    A = orc.kin3_matrix(p, -30.0)
    x0 = np.array([0.6, 0.3, 0.1])
    T = 2.0
    exact = scipy.linalg.expm(T * A) @ x0
    errs = []
    for n in (200, 400, 800):
        x = x0.copy()
        for _ in range(n):
            x, _ = orc.kin_newton_n(A, T / n, x)
        errs.append(np.abs(x - exact).max())
    assert 1.8 < errs[0] / errs[1] < 2.2 and 1.8 < errs[1] / errs[2] < 2.2


# ------------------------------------------------------------------ P13

def decay(rate_dt, n):
    """(1 + rate_dt)^-n and 1 - (1 + rate_dt)^-n without cancellation."""
    q = -n * math.log1p(rate_dt)
    return math.exp(q), -math.expm1(q)


def cacum(k=0.5182, tau=200.0, cai0=5e-5, kf=100.0, kb=0.1, btot=0.05):
    return np.array([k, tau, cai0, kf, kb, btot])


def test_p13_rest_is_a_fixed_point(orc):
    p = cacum()
    s = orc.mech_init(W.TYPE_CACUM, p, np.zeros(1, np.int32), np.array([-65.0]))
    y, it = orc.cacum_newton(p, 0.025, 0.0, s[:, 0])
    assert abs(y[0] - s[0, 0]) <= 1e-19 and abs(y[1] - s[1, 0]) <= 1e-18
    assert it == 1


def test_p13_unbuffered_closed_form(orc):
    p = cacum(kf=0.0, kb=0.0)
    ica, dt, N = -2e-3, 0.025, 400
    cstar = p[2] - p[0] * ica * p[1]
    x = np.array([1e-4, 0.0])
    for _ in range(N):
        x, _ = orc.cacum_newton(p, dt, ica, x)
    f, g = decay(dt / p[1], N)
    ref = 1e-4 * f + cstar * g
    assert x[0] == pytest.approx(ref, rel=1e-13)


def test_p13_unbinding_closed_form(orc):
    p = cacum(kf=0.0, kb=0.3, tau=1e300)
    dt, N = 0.025, 300
    x = np.array([2e-4, 1e-3])
    for _ in range(N):
        x, _ = orc.cacum_newton(p, dt, 0.0, x)
    cab = 1e-3 * decay(dt * 0.3, N)[0]
    assert x[1] == pytest.approx(cab, rel=1e-13)
    assert x[0] == pytest.approx(2e-4 + 1e-3 - cab, rel=1e-13)


def test_p13_binding_conserves_total_calcium(orc):
    p = cacum(tau=1e300)
    dt = 0.025
    x = np.array([3e-3, 1e-2])
    tot = x.sum()
    for _ in range(100):
        x, _ = orc.cacum_newton(p, dt, 0.0, x)
    assert x.sum() == pytest.approx(tot, rel=1e-14)
    # an inward current adds k |ica| dt per step to the total
    ica = -0.01
    y, _ = orc.cacum_newton(p, dt, ica, x)
    assert y.sum() - x.sum() == pytest.approx(-p[0] * ica * dt, rel=1e-10)


def test_p13_irreversible_binding_drains_free_calcium(orc):
    p = cacum(kb=0.0, tau=1e300)
    x = np.array([1e-3, 0.0])
    for _ in range(20000):
        x, _ = orc.cacum_newton(p, 0.025, 0.0, x)
    assert x[0] < 1e-12 and x[1] == pytest.approx(1e-3, rel=1e-12)


def test_p13_newton_converges_quadratically(orc):
    """e_{k+1} <= C e_k^2 with a constant C (~25 here); a Jacobian with a
    dropped or wrong term converges only linearly and fails this."""
    p = cacum(kf=2000.0)
    x = np.array([1e-2, 0.0])
    dt, ica = 0.1, -0.2
    ys = [orc.cacum_newton(p, dt, ica, x, tol=0.0, max_iter=k)[0] for k in range(1, 9)]
    ystar = ys[-1]
    e = [np.abs(y - ystar).max() for y in ys[:4]]
    assert e[0] > 1e-4
    for a, b in zip(e, e[1:]):
        assert b <= 100.0 * a * a
    _, it = orc.cacum_newton(p, dt, ica, x)
    assert it <= 6
    # the physical root: free and bound calcium nonnegative, buffer not overfull
    assert ystar[0] >= 0 and 0 <= ystar[1] <= p[5]


def test_p13_agrees_with_fsolve(orc):
    p = cacum(kf=300.0, kb=0.05)
    x = np.array([4e-3, 1e-2])
    dt, ica = 0.2, -1.0
    k, tau, cai0, kf, kb, btot = p

    def F(y):
        bind = kf * y[0] * (btot - y[1]) - kb * y[1]
        return [y[0] - x[0] - dt * (-k * ica - bind - (y[0] - cai0) / tau),
                y[1] - x[1] - dt * bind]

    ref = scipy.optimize.fsolve(F, x, xtol=1e-14)
    y, _ = orc.cacum_newton(p, dt, ica, x)
    np.testing.assert_allclose(y, ref, rtol=1e-10)


# ------------------------------------------------------------------ P14

def test_p14_hh_splits_into_sodium_and_potassium(orc):
    p = W.hh_params()
    rng = np.random.default_rng(14)
    n = 64
    ni = np.arange(n, dtype=np.int32)
    v = rng.uniform(-90, 40, n)
    v[0], v[1] = p[3], p[4]  # at ena and at ek
    s = rng.uniform(0.01, 1, (3, n))
    ion = orc.mech_ion_cur(W.TYPE_HH, p, ni, v, s, n)
    c, _ = orc.mech_currents(W.TYPE_HH, p, ni, v, s)
    np.testing.assert_allclose(ion[1] + ion[2] + p[2] * (v - p[5]), c, rtol=1e-13,
                               atol=1e-16)
    assert ion[1][0] == 0.0 and ion[2][1] == 0.0
    below = v < p[3]
    assert np.all(ion[1][below] < 0) and np.all(ion[3] == 0)


def test_p14_tagged_channel_writes_node_sums(orc):
    net = W.cortical_mix(200, seed=14)
    rng = np.random.default_rng(3)
    for m in net["mechs"]:
        ns = orc.n_states(m["type"], m["params"])
        s = rng.uniform(0, 1, (ns, m["node_index"].size))
        c, _ = orc.mech_currents(m["type"], m["params"], m["node_index"], net["v0"], s)
        ref = np.zeros(200)
        np.add.at(ref, m["node_index"], c)
        for ion in (1, 2, 3):
            got = orc.mech_ion_cur(m["type"], m["params"], m["node_index"], net["v0"], s,
                                   200, ion=ion)
            np.testing.assert_allclose(got[ion], ref, rtol=1e-13, atol=1e-300)
            assert np.all(np.delete(got, ion, axis=0) == 0)
        none = orc.mech_ion_cur(m["type"], m["params"], m["node_index"], net["v0"], s, 200)
        assert np.all(none == 0)


def test_p14_calcium_path_closed_form(orc):
    """A non-gated calcium conductance writes ica = g (v - eca) at clamped
    v; the unbuffered accumulation then has a closed form over N steps."""
    n = 5
    v = np.linspace(-70, 10, n)
    ni = np.arange(n, dtype=np.int32)
    gca, eca = 2e-4, 120.0
    chan = W.cnexp_params(gca, eca, [])
    buf = cacum(kf=0.0, kb=0.0)
    mechs = [dict(type=W.TYPE_CNEXP, params=chan, node_index=ni, ion=W.ION_CA),
             dict(type=W.TYPE_CACUM, params=buf, node_index=ni)]
    s_buf = np.vstack([np.full(n, buf[2]), np.zeros(n)])  # no buffer: cab = 0
    dt, N = 0.025, 300
    vv, rhs, d, ion, st = orc.step_ions(mechs, [np.zeros((0, n)), s_buf], v, n, dt,
                                        nsteps=N, clamp_v=True)
    ica = gca * (v - eca)
    np.testing.assert_allclose(ion[3], ica, rtol=1e-15)
    assert np.all(ion[1] == 0) and np.all(ion[2] == 0)
    cstar = buf[2] - buf[0] * ica * buf[1]
    f, g = decay(dt / buf[1], N)
    ref = buf[2] * f + cstar * g
    np.testing.assert_allclose(st[1][0], ref, rtol=1e-13)
    assert np.all(vv == v)


def test_p14_ion_recording_leaves_membrane_path_unchanged(orc):
    net = W.cortical_ions(150, seed=9, kin3_frac=0.6)
    mechs = [m for m in net["mechs"] if m["type"] != W.TYPE_CACUM]
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], net["v0"]) for m in mechs]
    a = orc.step(mechs, st, net["v0"], 150, 0.025, nsteps=7)
    b = orc.step_ions(mechs, st, net["v0"], 150, 0.025, nsteps=7)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y)
    for x, y in zip(a[3], b[4]):
        assert np.array_equal(x, y)
    # with every current tagged, the ion arrays add up to the membrane
    # current of the step: -rhs == ina + ik + ica
    tagged = [m for m in mechs if m["ion"] != W.ION_NONE]
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], net["v0"]) for m in tagged]
    _, rhs, _, ion, _ = orc.step_ions(tagged, st, net["v0"], 150, 0.025, nsteps=3)
    scale = np.abs(ion).sum(axis=0) + 1e-300
    assert np.all(np.abs(-rhs - ion[1:].sum(axis=0)) <= 1e-13 * scale)
    assert np.abs(ion[1]).max() > 0 and np.abs(ion[2]).max() > 0 and np.abs(ion[3]).max() > 0
