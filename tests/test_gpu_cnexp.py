"""GPU parity of the cnexp family (HH and generic gates) against the FP64
oracle, through the C ABI: state, INITIAL, current accumulation, the fused
and generic network step, mixed precision, and full-size sampled parity."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import (TOL_FP64, make_mechs, node_scale, state_err,
                         sub_network, to_dev)

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _ctx(api, **kw):
    return api.Context(0, **kw)


def _random_states(wl, seed):
    rng = np.random.default_rng(seed)
    from oracle import oracle as orc
    return [rng.uniform(0, 1, size=(orc.n_states(m["type"], m["params"]),
                                    m["node_index"].size)) for m in wl["mechs"]]


def _wl_hh(n=4099, seed=1):
    wl = W.hh_single(n, seed)
    wl["v0"] = W.Stream(seed, 9).uniform(n, -100.0, 60.0)
    return wl


# ---------------------------------------------------------------- state

@pytest.mark.parametrize("which", ["hh", "mix"])
@pytest.mark.parametrize("dt", [0.025, 0.3])
def test_state_one_step_fp64(api, orc, which, dt):
    wl = _wl_hh() if which == "hh" else W.cortical_mix(3001, seed=5, v_lo=-100, v_hi=60)
    ctx = _ctx(api)
    mechs = make_mechs(ctx, wl)
    st0 = _random_states(wl, 3)
    v = to_dev(wl["v0"])
    for m, s, spec in zip(mechs, st0, wl["mechs"]):
        if m.n_states == 0:
            continue
        m.set_states(to_dev(s))
        m.state(dt, v)
        got = m.states().cpu().numpy()
        ref = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                             wl["v0"], s, dt)
        assert state_err(got, ref) <= TOL_FP64, (spec.get("name"), state_err(got, ref))
    assert ctx.sync() == 0


def test_init_fp64(api, orc):
    wl = W.cortical_mix(2003, seed=6, v_lo=-100, v_hi=60)
    wl["mechs"].insert(0, _wl_hh(2003)["mechs"][0])
    ctx = _ctx(api)
    mechs = make_mechs(ctx, wl)
    v = to_dev(wl["v0"])
    for m, spec in zip(mechs, wl["mechs"]):
        m.init(v)
        ref = orc.mech_init(spec["type"], spec["params"], spec["node_index"], wl["v0"])
        assert state_err(m.states().cpu().numpy(), ref) <= TOL_FP64


def test_vtrap_singular_point(api, orc):
    # v exactly at the LINOID singularity of alpha_m (-40) and alpha_n (-55)
    v0 = np.array([-40.0, -55.0, -40.0 + 1e-7, -55.0 - 3e-6, -65.0])
    ni = np.arange(5, dtype=np.int32)
    wl = dict(n_nodes=5, mechs=[dict(type=W.TYPE_HH, params=W.hh_params(), node_index=ni)])
    ctx = _ctx(api)
    (m,) = make_mechs(ctx, wl)
    v = to_dev(v0)
    s0 = np.full((3, 5), 0.3)
    m.set_states(to_dev(s0))
    m.state(0.025, v)
    ref = orc.mech_state(W.TYPE_HH, W.hh_params(), ni, v0, s0, 0.025)
    assert state_err(m.states().cpu().numpy(), ref) <= TOL_FP64
    assert ctx.sync() == 0


# ------------------------------------------------------------------ cur

def _cur_case(api, orc, wl, seed=4):
    ctx = _ctx(api)
    mechs = make_mechs(ctx, wl)
    st = _random_states(wl, seed)
    rng = np.random.default_rng(seed)
    n = wl["n_nodes"]
    rhs0 = rng.normal(size=n)
    d0 = rng.uniform(0.05, 1.0, size=n)
    v = to_dev(wl["v0"])
    rhs, d = to_dev(rhs0), to_dev(d0)
    r_ref, d_ref = rhs0.copy(), d0.copy()
    for m, s, spec in zip(mechs, st, wl["mechs"]):
        m.set_states(to_dev(s))
        m.cur(v, rhs, d)
        r_ref, d_ref = orc.mech_cur(spec["type"], spec["params"], spec["node_index"],
                                    wl["v0"], s, r_ref, d_ref)
    sr, sd = node_scale(orc, wl, st, wl["v0"], rhs0, d0)
    er = np.abs(rhs.cpu().numpy() - r_ref)
    ed = np.abs(d.cpu().numpy() - d_ref)
    assert np.all(er <= TOL_FP64 * sr + 1e-300), float(np.max(er / np.maximum(sr, 1e-300)))
    assert np.all(ed <= TOL_FP64 * sd + 1e-300)
    # untouched nodes stay bitwise unchanged
    touched = np.zeros(n, bool)
    for spec in wl["mechs"]:
        touched[spec["node_index"]] = True
    assert np.array_equal(rhs.cpu().numpy()[~touched], rhs0[~touched])
    # determinism: a second accumulation from the same start is bitwise equal
    rhs2, d2 = to_dev(rhs0), to_dev(d0)
    for m in mechs:
        m.cur(v, rhs2, d2)
    assert torch.equal(rhs, rhs2) and torch.equal(d, d2)
    assert ctx.sync() == 0


def test_cur_mix(api, orc):
    _cur_case(api, orc, W.cortical_mix(4001, seed=7, v_lo=-100, v_hi=60))


def test_cur_hh(api, orc):
    _cur_case(api, orc, _wl_hh(1000))


def test_cur_long_segments(api, orc):
    """Segments longer than a warp and straddling several 32-wide pieces."""
    s = W.Stream(11, 1)
    lens = s.integers(300, 0, 100)
    lens[5] = 257
    lens[6] = 31
    lens[7] = 33
    ni = np.repeat(np.arange(300), lens).astype(np.int32)
    blocks = W.cortical_type_params(2)
    wl = dict(n_nodes=300, v0=s.uniform(300, -90, 40),
              mechs=[dict(type=W.TYPE_CNEXP, params=blocks[0], node_index=ni),
                     dict(type=W.TYPE_CNEXP, params=blocks[9],
                          node_index=np.array([3, 3, 299], dtype=np.int32))])
    _cur_case(api, orc, wl)


def test_empty_mechanism(api, orc):
    ctx = _ctx(api)
    from paper_1905_02241_b300.api import Mechanism
    m = Mechanism(ctx, W.TYPE_CNEXP, np.zeros(0, np.int32), 10, W.cortical_type_params(2)[0])
    v = to_dev(np.full(10, -65.0))
    rhs, d = to_dev(np.zeros(10)), to_dev(np.zeros(10))
    m.init(v)
    m.state(0.025, v)
    m.cur(v, rhs, d)
    ctx.step([m], 0.025, 1.0, v, rhs, d, 3)
    assert float(rhs.abs().sum()) == 0.0
    np.testing.assert_allclose(d.cpu().numpy(), 1e-3 / 0.025)
    assert ctx.sync() == 0


# ----------------------------------------------------------------- step

def _step_case(api, orc, wl, nsteps, tol, fused=None, **opts):
    ctx = _ctx(api, **opts)
    mechs = make_mechs(ctx, wl)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    for m, s in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(s))
    n = wl["n_nodes"]
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, nsteps)
    assert ctx.sync() == 0
    if fused is not None:  # the path the tile budget selects: fused tiles or generic
        plan = ctx.plan(mechs)
        assert plan["fused"] == fused and (not fused or plan["tiles"] > 1), plan
    v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], st0, wl["v0"], n, 0.025,
                                          nsteps=nsteps, clamp_v=opts.get("clamp_v", 0))
    ev = np.max(np.abs(v.cpu().numpy() - v_ref) / np.maximum(np.abs(v_ref), 1.0))
    es = max([state_err(m.states().cpu().numpy(), s) for m, s in zip(mechs, s_ref)
              if m.n_states] + [0.0])
    # rhs/d of the last step.  sum|g (v - e)| <= d * 200 mV bounds the sum of
    # the magnitudes of rhs's terms, so it is a cancellation-safe scale.
    er = np.max(np.abs(rhs.cpu().numpy() - r_ref) / (200.0 * d_ref))
    ed = np.max(np.abs(d.cpu().numpy() - d_ref) / np.abs(d_ref))
    assert ev <= tol and es <= tol and er <= tol and ed <= tol, (ev, es, er, ed)
    return ev, es


@pytest.mark.parametrize("tile_smem", [0, 16384, 64])  # 64: no tile fits -> generic
def test_step_one_fp64(api, orc, tile_smem):
    wl = W.cortical_mix(5003, seed=8)
    _step_case(api, orc, wl, 1, TOL_FP64, fused=tile_smem != 64, tile_smem=tile_smem)


@pytest.mark.parametrize("window,use_graph", [(40, 1), (7, 0), (3, 1)])
def test_step_window_fp64(api, orc, window, use_graph):
    wl = W.cortical_mix(3001, seed=9)
    _step_case(api, orc, wl, 20, 1e-10, fused=True, window=window, use_graph=use_graph,
               tile_smem=16384)


def test_step_hh_trajectory(api, orc):
    """HH on 4096 isolated nodes for 1000 steps (25 ms): trajectory parity."""
    wl = W.hh_single(4096, 1)
    ev, es = _step_case(api, orc, wl, 1000, 1e-9)
    print(f"HH 1000-step trajectory: max rel v err {ev:.2e}, state err {es:.2e}")


def test_step_clamped(api, orc):
    wl = W.cortical_mix(2001, seed=10)
    _step_case(api, orc, wl, 5, 1e-11, clamp_v=1)


def test_step_with_hh_and_mix(api, orc):
    wl = W.cortical_mix(2500, seed=12)
    wl["mechs"].insert(3, dict(type=W.TYPE_HH, params=W.hh_params(),
                               node_index=np.arange(0, 2500, 3, dtype=np.int32)))
    _step_case(api, orc, wl, 10, 1e-10, fused=True, tile_smem=24576)


# ------------------------------------------------------------ precision

def test_step_crowded_node_beyond_the_slot_range(api, orc):
    """A node carrying more currents than a tile can number with its uint16
    slots (70,000 instances of one type on node 0 of a 40-node network): no
    tile fits that node, so the step falls back to the per-mechanism launches
    (one warp reduces the whole segment), which match the oracle."""
    wl = W.cortical_mix(40, seed=31)
    wl["mechs"].append(dict(type=W.TYPE_CNEXP, params=W.cortical_type_params(2)[4],
                            node_index=np.zeros(70000, dtype=np.int32)))
    _step_case(api, orc, wl, 3, 1e-10, fused=False)


def test_mixed_precision_errors(api, orc):
    """MIXED vs the FP64 oracle, per quantity (one step and 200 steps)."""
    wl = W.cortical_mix(3001, seed=13)
    n = wl["n_nodes"]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    out = {}
    for nsteps in (1, 200):
        ctx = _ctx(api, precision=api.NMODL_MIXED, tile_smem=24576)
        mechs = make_mechs(ctx, wl)
        for m, s in zip(mechs, st0):
            if m.n_states:
                m.set_states(to_dev(s))
        v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
        ctx.step(mechs, 0.025, 1.0, v, rhs, d, nsteps)
        assert ctx.sync() == 0
        plan = ctx.plan(mechs)
        assert plan["fused"] and plan["tiles"] > 1, plan
        v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], st0, wl["v0"], n, 0.025,
                                              nsteps=nsteps)
        es = max(float(np.max(np.abs(m.states().cpu().numpy() - s)))
                 for m, s in zip(mechs, s_ref) if m.n_states)
        ev = float(np.max(np.abs(v.cpu().numpy() - v_ref)))
        ed = float(np.max(np.abs(d.cpu().numpy() - d_ref) / d_ref))
        out[nsteps] = (es, ev, ed)
    print("MIXED errors (states abs, v abs mV, d rel):", out)
    assert out[1][0] <= 1e-6 and out[1][1] <= 1e-5 and out[1][2] <= 1e-6
    assert out[200][0] <= 1e-4 and out[200][1] <= 1e-2


def test_mixed_step_with_hh_and_mix(api, orc):
    """MIXED fused step with HH among the cnexp types (an HH instance takes
    three node-major slots, one per current) against the FP64 oracle, per
    quantity, 20 steps on many tiles."""
    wl = W.cortical_mix(2500, seed=12)
    wl["mechs"].insert(3, dict(type=W.TYPE_HH, params=W.hh_params(),
                               node_index=np.arange(0, 2500, 3, dtype=np.int32)))
    n = wl["n_nodes"]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    ctx = _ctx(api, precision=api.NMODL_MIXED, tile_smem=24576)
    mechs = make_mechs(ctx, wl)
    for m, s in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(s))
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 20)
    assert ctx.sync() == 0
    plan = ctx.plan(mechs)
    assert plan["fused"] and plan["tiles"] > 1, plan
    v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], st0, wl["v0"], n, 0.025, nsteps=20)
    es = max(float(np.max(np.abs(m.states().cpu().numpy() - s)))
             for m, s in zip(mechs, s_ref) if m.n_states)
    ev = float(np.max(np.abs(v.cpu().numpy() - v_ref)))
    ed = float(np.max(np.abs(d.cpu().numpy() - d_ref) / d_ref))
    er = float(np.max(np.abs(rhs.cpu().numpy() - r_ref) / (200.0 * d_ref)))
    print("MIXED with HH, 20 steps (states abs, v abs mV, d rel, rhs):", es, ev, ed, er)
    assert es <= 2e-5 and ev <= 2e-3 and ed <= 1e-6 and er <= 1e-6


def test_mixed_standalone_state(api, orc):
    wl = W.cortical_mix(2001, seed=14, v_lo=-100, v_hi=60)
    ctx = _ctx(api, precision=api.NMODL_MIXED)
    mechs = make_mechs(ctx, wl)
    st0 = _random_states(wl, 5)
    v = to_dev(wl["v0"])
    worst = 0.0
    for m, s, spec in zip(mechs, st0, wl["mechs"]):
        if not m.n_states:
            continue
        m.set_states(to_dev(s))
        m.state(0.025, v)
        ref = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                             wl["v0"], s, 0.025)
        worst = max(worst, float(np.max(np.abs(m.states().cpu().numpy() - ref))))
    print("MIXED standalone state abs err", worst)
    assert worst <= 1e-6


# -------------------------------------------------- full-size, sampled

def test_full_size_sampled_parity(api, orc):
    """2M-node cortical mix in the launch configuration the benchmark uses
    (fused FP64 step, 40-step graph windows): 200 steps on the GPU, checked
    on 1500 sampled nodes that the oracle integrates as their own isolated
    sub-network."""
    wl = W.cortical_mix(2_000_000, seed=2)
    ctx = _ctx(api)
    mechs = make_mechs(ctx, wl)
    n = wl["n_nodes"]
    v = to_dev(wl["v0"])
    for m in mechs:
        m.init(v)
    rhs, d = to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 200)
    assert ctx.sync() == 0
    nodes = np.unique(W.Stream(77, 1).integers(1500, 0, n - 1))
    sub, sel = sub_network(wl, nodes)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"][nodes])
           for m in sub["mechs"]]
    v_ref, r_ref, d_ref, s_ref = orc.step(sub["mechs"], st0, wl["v0"][nodes], nodes.size,
                                          0.025, nsteps=200)
    vg = v.cpu().numpy()[nodes]
    assert np.max(np.abs(vg - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-9
    for m, s, idx in zip(mechs, s_ref, sel):
        if m.n_states:
            g = m.states().cpu().numpy()[:, idx]
            assert state_err(g, s) <= 1e-9
    np.testing.assert_allclose(d.cpu().numpy()[nodes], d_ref, rtol=1e-9)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_full_size_sampled_parity(api, orc, prec):
    """The batched benchmark's configuration: 64 networks of uneven size
    (~8.5M nodes, ~104M instances) in one fused launch per 40-step window
    with CUDA graphs and the autotuned plan, 200 steps, checked on 1,500
    sampled nodes that the oracle integrates as their own sub-network (FP64
    at the trajectory tolerance; MIXED within its 200-step bounds)."""
    wl = W.batched_networks(64, seed=3)
    P = api.NMODL_FP64 if prec == "fp64" else api.NMODL_MIXED
    ctx = _ctx(api, precision=P)
    mechs = make_mechs(ctx, wl)
    n = wl["n_nodes"]
    v = to_dev(wl["v0"])
    for m in mechs:
        m.init(v)
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 200)
    assert ctx.sync() == 0
    assert ctx.plan(mechs)["fused"]
    nodes = np.unique(W.Stream(79, 1).integers(1500, 0, n - 1))
    sub, sel = sub_network(wl, nodes)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"][nodes])
           for m in sub["mechs"]]
    v_ref, r_ref, d_ref, s_ref = orc.step(sub["mechs"], st0, wl["v0"][nodes], nodes.size,
                                          0.025, nsteps=200)
    vg = v.cpu().numpy()[nodes]
    gs = [m.states()[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy() if m.n_states
          else None for m, idx in zip(mechs, sel)]
    if prec == "fp64":
        assert np.max(np.abs(vg - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-9
        for g, s in zip(gs, s_ref):
            if g is not None:
                assert state_err(g, s) <= 1e-9
        np.testing.assert_allclose(d.cpu().numpy()[nodes], d_ref, rtol=1e-9)
    else:
        assert np.max(np.abs(vg - v_ref)) <= 1e-2
        for g, s in zip(gs, s_ref):
            if g is not None:
                assert np.max(np.abs(g - s)) <= 1e-4


def test_table_exp_ulp_error():
    """The FP64 exp of the state kernels (Tang's table-driven method, 2048-entry
    table, degree-3 polynomial) against mpmath at 40 digits and against
    CUDA's exp: within 1.5 ulp (table entries are rounded to double)."""
    import mpmath
    from paper_1905_02241_b300 import _lib
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    x = np.concatenate([rng.uniform(-708, 708, 20000), rng.uniform(-1, 1, 20000),
                        rng.uniform(-30, 30, 20000), [0.0, -0.0, 1e-300, 707.9, -707.9]])
    xd = to_dev(x)
    y = torch.empty_like(xd)
    yc = torch.empty_like(xd)
    _lib.nmodl_math_eval(0, x.size, xd.data_ptr(), y.data_ptr(), 0)
    _lib.nmodl_math_eval(1, x.size, xd.data_ptr(), yc.data_ptr(), 0)
    torch.cuda.synchronize()
    y, yc = y.cpu().numpy(), yc.cpu().numpy()
    idx = np.random.default_rng(4).choice(x.size, 3000, replace=False)
    worst = 0.0
    for i in idx:
        ref = mpmath.exp(mpmath.mpf(float(x[i])))
        ulp = np.spacing(float(ref))
        worst = max(worst, abs(float(mpmath.mpf(float(y[i])) - ref)) / ulp)
    print(f"table exp: max error {worst:.3f} ulp (3000 samples vs mpmath)")
    assert worst <= 1.5
    assert np.max(np.abs(y - yc) / np.abs(yc)) <= 5e-16


def test_fast_reciprocal_within_one_ulp():
    """The reciprocal of the gate and node updates (hardware approximation +
    one third-order Newton step) against the correctly rounded 1/x: within
    one ulp over normal-range inputs, exact at powers of two."""
    from paper_1905_02241_b300 import _lib
    rng = np.random.default_rng(7)
    x = np.concatenate([rng.uniform(0.5, 2.0, 100000),
                        rng.uniform(1, 10, 50000) * 10.0 ** rng.integers(-300, 300, 50000),
                        -rng.uniform(1e-6, 1e6, 20000), 2.0 ** np.arange(-1000, 1000, 37)])
    xd = to_dev(x)
    y = torch.empty_like(xd)
    _lib.nmodl_math_eval(3, x.size, xd.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    got, ref = y.cpu().numpy(), 1.0 / x
    ulps = np.abs(got - ref) / np.spacing(np.abs(ref))
    print(f"fast reciprocal: max {ulps.max():.3f} ulp, exact {np.mean(got == ref):.4f}")
    assert ulps.max() <= 1.0
    p2 = x.size - np.arange(-1000, 1000, 37).size
    assert np.array_equal(got[p2:], ref[p2:])


def test_rate_denominators_one_plus_minus_exp():
    """The SIGMOID and LINOID denominators 1 + e^x and 1 - e^x (the exp's
    constant part 1 +- 2^m T formed by integer operations, then one fma)
    against mpmath: 1 + e^x within 2 ulp; 1 - e^x within 2 ulp of e^x plus
    one of the result (the cancellation near x = 0 amplifies e^x's own
    error, as in 1 - exp(x) itself)."""
    import mpmath
    from paper_1905_02241_b300 import _lib
    mpmath.mp.dps = 40
    rng = np.random.default_rng(13)
    x = np.concatenate([rng.uniform(-700, 700, 4000), rng.uniform(-40, 40, 8000),
                        rng.uniform(-1, 1, 4000), [0.0, 1e-9, -1e-9, 36.7, 37.3, 38.2,
                                                   -36.7, -745.0, 709.0]])
    xd = to_dev(x)
    yp, ym = torch.empty_like(xd), torch.empty_like(xd)
    _lib.nmodl_math_eval(5, x.size, xd.data_ptr(), yp.data_ptr(), 0)
    _lib.nmodl_math_eval(6, x.size, xd.data_ptr(), ym.data_ptr(), 0)
    torch.cuda.synchronize()
    yp, ym = yp.cpu().numpy(), ym.cpu().numpy()
    worst_p = worst_m = 0.0
    for i in range(x.size):
        e = mpmath.exp(mpmath.mpf(float(x[i])))
        rp, rm = 1 + e, 1 - e
        if mpmath.isinf(rp) or float(rp) == float("inf"):
            assert np.isinf(yp[i]) and np.isinf(ym[i])
            continue
        worst_p = max(worst_p, float(abs(mpmath.mpf(float(yp[i])) - rp)) / np.spacing(float(rp)))
        bound = 2 * np.spacing(float(e)) + np.spacing(abs(float(rm)))
        worst_m = max(worst_m, float(abs(mpmath.mpf(float(ym[i])) - rm)) / bound)
    print(f"1 + e^x: max {worst_p:.3f} ulp; 1 - e^x: max {worst_m:.3f} of the bound")
    assert worst_p <= 2.0
    assert worst_m <= 1.0


def test_fast_division_within_one_ulp():
    """The division of the gate updates (a quotient formed in single
    precision, corrected by one FP64 residual step) against the correctly
    rounded quotient: within one ulp over normal-range operands of both
    signs, exact when both are powers of two; zero numerators, huge or tiny
    operands and quotients near the range ends take IEEE division."""
    from paper_1905_02241_b300 import _lib
    rng = np.random.default_rng(11)
    n = 200000
    a = rng.uniform(1, 10, n) * 10.0 ** rng.integers(-150, 150, n) * rng.choice([-1, 1], n)
    b = rng.uniform(1, 10, n) * 10.0 ** rng.integers(-150, 150, n) * rng.choice([-1, 1], n)
    a[:500] = 2.0 ** rng.integers(-300, 300, 500)
    b[:500] = -(2.0 ** rng.integers(-300, 300, 500))
    special = np.array([[0.0, 3.0], [-0.0, 2.0], [1e308, 1e-10], [1e-310, 3.0], [5.0, 1e-320],
                        [1e300, 1e-300], [1.5, 1e308], [7.0, 7.0]])
    a = np.concatenate([a, special[:, 0]])
    b = np.concatenate([b, special[:, 1]])
    xd = to_dev(np.stack([a, b], axis=1).reshape(-1))
    y = torch.empty(a.size, dtype=torch.float64, device="cuda")
    _lib.nmodl_math_eval(4, a.size, xd.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    with np.errstate(over="ignore", divide="ignore"):
        ref = a / b
    got = y.cpu().numpy()
    fin = np.isfinite(ref) & (ref != 0)
    ulps = np.abs(got[fin] - ref[fin]) / np.spacing(np.abs(ref[fin]))
    print(f"fast division: max {ulps.max():.3f} ulp, correctly rounded {np.mean(got == ref):.4f}")
    assert ulps.max() <= 1.0
    assert np.array_equal(got[:500], ref[:500])
    assert np.array_equal(got[n:], ref[n:])   # out-of-line IEEE division


def test_integer_pipe_conversions_round_like_hardware():
    """double -> float -> double through the integer-pipe conversions equals
    numpy's float32 rounding bit for bit (ties, carries into the exponent,
    zeros, subnormal, huge, infinite and NaN values included)."""
    from paper_1905_02241_b300 import _lib
    rng = np.random.default_rng(5)
    f = rng.uniform(-1, 1, 20000).astype(np.float32).astype(np.float64)
    ulp = np.spacing(np.abs(f).astype(np.float32)).astype(np.float64)
    x = np.concatenate([
        rng.uniform(-1, 1, 50000), rng.uniform(0, 1, 50000) * 10.0 ** rng.integers(-40, 40, 50000),
        f + 0.5 * ulp, f - 0.5 * ulp, f + 0.5 * ulp * (1 + 2e-16),   # ties and near-ties
        [0.0, -0.0, 1e-300, -1e-310, 3.4028234663852886e38, 3.5e38, 1.1754943508222875e-38,
         1.0 - 2 ** -25, 2.0 - 2 ** -24, np.inf, -np.inf, np.nan, 1.4e-45, -2.9e-39]])
    xd = to_dev(x)
    y = torch.empty_like(xd)
    _lib.nmodl_math_eval(2, x.size, xd.data_ptr(), y.data_ptr(), 0)
    torch.cuda.synchronize()
    with np.errstate(over="ignore"):
        ref = x.astype(np.float32).astype(np.float64)
    got = y.cpu().numpy()
    same = (got == ref) | (np.isnan(got) & np.isnan(ref))
    assert same.all(), x[~same][:5]
    assert np.array_equal(np.signbit(got), np.signbit(ref))


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_resume_is_bitwise(api, prec):
    """Save states and v mid-run (nmodl_get_state), restore them into a new
    context (nmodl_set_state) and continue: the continuation is bitwise equal
    to the uninterrupted run."""
    p = api.NMODL_FP64 if prec == "fp64" else api.NMODL_MIXED
    wl = W.cortical_mix(3001, seed=15)
    n = wl["n_nodes"]
    ctx = _ctx(api, precision=p)
    mechs = make_mechs(ctx, wl)
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    for m in mechs:
        m.init(v)
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 40)
    ckpt_v = v.clone()
    ckpt = [m.states().clone() for m in mechs]
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 40)
    ref_v, ref_s = v.clone(), [m.states() for m in mechs]
    ctx2 = _ctx(api, precision=p)
    mechs2 = make_mechs(ctx2, wl)
    for m, s in zip(mechs2, ckpt):
        if m.n_states:
            m.set_states(s)
    v2, rhs2, d2 = ckpt_v.clone(), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx2.step(mechs2, 0.025, 1.0, v2, rhs2, d2, 40)
    assert torch.equal(v2, ref_v)
    for m, s in zip(mechs2, ref_s):
        assert torch.equal(m.states(), s)
    assert ctx.sync() == 0 and ctx2.sync() == 0


@pytest.mark.parametrize("fused", [True, False])
def test_pade_cnexp_parity(api, orc, fused):
    """(1,1) Pade cnexp (Section 5.2 option) against the oracle's Pade mode:
    one-step states at 1e-12 and 20 network steps, fused and standalone."""
    wl = W.cortical_mix(2001, seed=16, v_lo=-100, v_hi=60)
    opts = dict(cnexp_pade=1) if fused else dict(cnexp_pade=1, tile_smem=64)
    ctx = _ctx(api, **opts)
    mechs = make_mechs(ctx, wl)
    st0 = _random_states(wl, 8)
    v = to_dev(wl["v0"])
    with orc.pade_mode():
        for m, s, spec in zip(mechs, st0, wl["mechs"]):
            if not m.n_states:
                continue
            m.set_states(to_dev(s))
            m.state(0.025, v)
            ref = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                                 wl["v0"], s, 0.025)
            assert state_err(m.states().cpu().numpy(), ref) <= TOL_FP64
        _step_case(api, orc, wl, 20, 1e-10, **opts)
