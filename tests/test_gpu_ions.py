"""GPU parity of the small systems and of the ion currents against the FP64
oracle: the 3-state scheme (stationary INITIAL, one-solve step in FP64, the
FP32 elimination + FP64 refinement form, current), the calcium buffer
(INITIAL, Newton step reading ica), the ion write-back of nmodl_cur (HH
split, tagged channels) and whole steps of the ion-tagged cortical network
with the buffer reading the same step's ica; error paths of the ion ABI."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import TOL_FP64, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def mech(api, ctx, m, n_nodes):
    return api.Mechanism(ctx, m["type"], m["node_index"], n_nodes, m["params"],
                         ion=m.get("ion", 0))


def kin3_case(n, seed=12, per_node=1):
    p = W.kin3_params(W.Stream(seed, 1))
    n_nodes = max(1, n // per_node)
    ni = np.sort(W.Stream(seed, 2).integers(n, 0, n_nodes - 1)).astype(np.int32) \
        if per_node > 1 else np.arange(n, dtype=np.int32)
    v = W.Stream(seed, 3).uniform(n_nodes, -100.0, 60.0)
    x = W.Stream(seed, 4).dirichlet(n, 3, 1.0) if n else np.zeros((3, 0))
    return dict(type=W.TYPE_KIN3, params=p, node_index=ni), v, x, n_nodes


# ---------------------------------------------------------------- KIN3

@pytest.mark.parametrize("n", [0, 1, 33, 5003])
def test_kin3_init_and_step_fp64(api, orc, n):
    spec, v, x, n_nodes = kin3_case(n)
    ctx = api.Context(0)
    m = mech(api, ctx, spec, n_nodes)
    vd = to_dev(v)
    m.init(vd)
    ref0 = orc.mech_init(W.TYPE_KIN3, spec["params"], spec["node_index"], v)
    got0 = m.states().cpu().numpy()
    assert state_err(got0, ref0) <= 1e-13
    for dt in (0.025, 0.5):
        m.set_states(to_dev(x))
        m.state(dt, vd)
        ref = orc.mech_state(W.TYPE_KIN3, spec["params"], spec["node_index"], v, x, dt)
        got = m.states().cpu().numpy()
        assert state_err(got, ref) <= TOL_FP64, state_err(got, ref)
        if n:
            assert np.max(np.abs(got.sum(axis=0) - x.sum(axis=0))) <= 1e-15
            assert got.min() >= 0
    st = m.stats()
    assert st["nonconverged"] == 0 and st["newton_max"] == (1 if n else 0)
    assert ctx.sync() == 0


def test_kin3_mixed_refinement(api, orc):
    spec, v, x, n_nodes = kin3_case(4099, seed=13)
    ctx = api.Context(0, precision=api.NMODL_MIXED)
    m = mech(api, ctx, spec, n_nodes)
    m.set_states(to_dev(x))
    m.state(0.025, to_dev(v))
    ref = orc.mech_state(W.TYPE_KIN3, spec["params"], spec["node_index"], v, x, 0.025)
    got = m.states().cpu().numpy()
    err = np.abs(got - ref).max()
    assert err <= 1e-6, err  # FP32 rates: the solved system differs at ~1e-7
    # the refined solution satisfies its own (FP32-rate) system to FP64
    # rounding, so the columns of J keep summing to one: total conserved
    assert np.max(np.abs(got.sum(axis=0) - x.sum(axis=0))) <= 1e-14
    st = m.stats()
    assert st["nonconverged"] == 0 and 2 <= st["newton_max"] <= 5
    assert ctx.sync() == 0


def test_kin3_current_segments(api, orc):
    spec, v, x, n_nodes = kin3_case(6000, seed=14, per_node=3)
    ctx = api.Context(0)
    m = mech(api, ctx, spec, n_nodes)
    m.set_states(to_dev(x))
    rhs0 = W.Stream(14, 9).uniform(n_nodes, -1, 1)
    d0 = W.Stream(14, 10).uniform(n_nodes, 0.1, 1)
    rhs, d = to_dev(rhs0), to_dev(d0)
    m.cur(to_dev(v), rhs, d)
    rr, dr = orc.mech_cur(W.TYPE_KIN3, spec["params"], spec["node_index"], v, x, rhs0, d0)
    c, g = orc.mech_currents(W.TYPE_KIN3, spec["params"], spec["node_index"], v, x)
    sr, sd = np.abs(rhs0).copy(), np.abs(d0).copy()
    np.add.at(sr, spec["node_index"], np.abs(c))
    np.add.at(sd, spec["node_index"], np.abs(g))
    assert np.all(np.abs(rhs.cpu().numpy() - rr) <= TOL_FP64 * sr)
    assert np.all(np.abs(d.cpu().numpy() - dr) <= TOL_FP64 * sd)
    assert ctx.sync() == 0


# --------------------------------------------------------------- CACUM

def cacum_case(n, seed=15):
    p = W.cacum_params()
    ni = np.arange(n, dtype=np.int32)
    ica = -np.abs(W.Stream(seed, 1).loguniform(n, 1e-4, 2.0)) if n else np.zeros(0)
    x = np.vstack([W.Stream(seed, 2).loguniform(n, 1e-5, 1e-1),
                   W.Stream(seed, 3).uniform(n, 0.0, p[5])]) if n else np.zeros((2, 0))
    return dict(type=W.TYPE_CACUM, params=p, node_index=ni), ica, x


@pytest.mark.parametrize("n", [1, 31, 4097])
def test_cacum_init_and_newton(api, orc, n):
    spec, ica, x = cacum_case(n)
    ctx = api.Context(0)
    m = mech(api, ctx, spec, n)
    ica_d = to_dev(ica)
    ctx.set_ions(ica=ica_d)
    m.init(to_dev(np.full(n, -65.0)))
    ref0 = orc.mech_init(W.TYPE_CACUM, spec["params"], spec["node_index"], np.full(n, -65.0))
    assert state_err(m.states().cpu().numpy(), ref0) <= 1e-14
    for dt in (0.025, 0.25):
        m.set_states(to_dev(x))
        m.state(dt, to_dev(np.zeros(n)))
        ref, it = orc.mech_state(W.TYPE_CACUM, spec["params"], spec["node_index"],
                                 np.zeros(n), x, dt, ica=ica, want_iters=True)
        got = m.states().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-12))
        assert err <= TOL_FP64, err  # relative to the state itself
    st = m.stats()
    assert st["nonconverged"] == 0
    assert abs(st["newton_max"] - int(it.max())) <= 1
    assert ctx.sync() == 0


@pytest.mark.parametrize("n", [1, 4097])
def test_cacum_mixed_refinement(api, orc, n):
    """The mixed buffer step (Newton updates in FP32, then refinements with
    the FP64 residual through the FP32 Jacobian) against the FP64 oracle: the
    refinement reaches the oracle's Newton solution at the FP64 tolerance,
    every instance within the refinement budget."""
    spec, ica, x = cacum_case(n)
    ctx = api.Context(0, precision=api.NMODL_MIXED)
    m = mech(api, ctx, spec, n)
    ctx.set_ions(ica=to_dev(ica))
    for dt in (0.025, 0.25):
        m.set_states(to_dev(x))
        m.state(dt, to_dev(np.zeros(n)))
        ref = orc.mech_state(W.TYPE_CACUM, spec["params"], spec["node_index"], np.zeros(n), x,
                             dt, ica=ica)
        got = m.states().cpu().numpy()
        err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-12))
        assert err <= TOL_FP64, err
    assert m.stats()["nonconverged"] == 0
    assert ctx.sync() == 0


def test_cacum_needs_an_ica_array(api):
    spec, ica, x = cacum_case(8)
    ctx = api.Context(0)
    m = mech(api, ctx, spec, 8)
    with pytest.raises(api.NmodlError) as e:
        m.state(0.025, to_dev(np.zeros(8)))
    assert e.value.status == -1
    ctx.set_ions(ica=to_dev(np.zeros(9)))  # wrong length for this node set
    with pytest.raises(api.NmodlError):
        m.state(0.025, to_dev(np.zeros(8)))
    ctx.set_ions(ica=to_dev(np.zeros(8)))
    m.init(to_dev(np.zeros(8)))
    m.state(0.025, to_dev(np.zeros(8)))
    assert ctx.sync() == 0


# ----------------------------------------------------------------- ions

def test_ion_tags_rejected_where_meaningless(api):
    ctx = api.Context(0)
    ni = np.arange(4, dtype=np.int32)
    hh = api.Mechanism(ctx, api.NMODL_HH, ni, 4, W.hh_params())
    with pytest.raises(api.NmodlError):
        hh.set_ion(api.NMODL_ION_CA)
    ca = api.Mechanism(ctx, api.NMODL_CACUM, ni, 4, W.cacum_params())
    with pytest.raises(api.NmodlError):
        ca.set_ion(api.NMODL_ION_K)
    ch = api.Mechanism(ctx, api.NMODL_CNEXP, ni, 4, W.cnexp_params(1e-3, 120.0, []))
    with pytest.raises(api.NmodlError):
        ch.set_ion(7)
    ch.set_ion(api.NMODL_ION_CA)
    from paper_1905_02241_b300 import _lib
    p3 = W.kin3_params(W.Stream(1, 1))
    ni_d = to_dev(ni)
    with pytest.raises(_lib.NmodlError) as e:
        _lib.nmodl_cur_noalloc(0, 0, api.NMODL_KIN3, 4, ni_d.data_ptr(), 4,
                               p3.ctypes.data, p3.size, 0, 4, 0, 0, 0)
    assert e.value.status == -9


def test_cur_writes_ion_currents(api, orc):
    net = W.cortical_ions(3000, seed=16)
    n = net["n_nodes"]
    v = net["v0"]
    ctx = api.Context(0)
    ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    ctx.set_ions(*ions)
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    d = torch.zeros_like(rhs)
    rng = np.random.default_rng(16)
    hh = dict(type=W.TYPE_HH, params=W.hh_params(), node_index=np.arange(n, dtype=np.int32))
    specs = [hh] + [m for m in net["mechs"] if m["type"] != W.TYPE_CACUM]
    ref = np.zeros((4, n))
    scale = np.zeros(n)
    vd = to_dev(v)
    for spec in specs:
        m = mech(api, ctx, spec, n)
        ns = orc.n_states(spec["type"], spec["params"])
        s = rng.uniform(0, 1, (ns, spec["node_index"].size))
        m.set_states(to_dev(s))
        m.cur(vd, rhs, d)
        ref += orc.mech_ion_cur(spec["type"], spec["params"], spec["node_index"], v, s, n,
                                ion=spec.get("ion", 0))
        c, _ = orc.mech_currents(spec["type"], spec["params"], spec["node_index"], v, s)
        np.add.at(scale, spec["node_index"], np.abs(c))
    got = np.vstack([np.zeros(n)] + [t.cpu().numpy() for t in ions])
    for q in (1, 2, 3):
        assert np.all(np.abs(got[q] - ref[q]) <= TOL_FP64 * (scale + 1e-300)), q
        assert np.abs(ref[q]).max() > 0
    assert ctx.sync() == 0


def _run_network(api, net, nsteps, precision=0, set_ions=True):
    n = net["n_nodes"]
    ctx = api.Context(0, precision=precision)
    ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    if set_ions:
        ctx.set_ions(*ions)
    ms = [mech(api, ctx, m, n) for m in net["mechs"]]
    v = to_dev(net["v0"])
    for m in ms:
        m.init(v)
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    d = torch.zeros_like(rhs)
    ctx.step(ms, 0.025, 1.0, v, rhs, d, nsteps)
    assert ctx.sync() == 0
    return ctx, ms, v, rhs, d, ions


def test_network_one_step_parity(api, orc):
    """One step from identical FP64 inputs: v, rhs, d, ion currents and every
    state (including the buffer, which reads this step's ica)."""
    net = W.cortical_ions(4000, seed=17)
    n = net["n_nodes"]
    ctx, ms, v, rhs, d, ions = _run_network(api, net, 1)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], net["v0"])
           for m in net["mechs"]]
    vr, rr, dr, ir, sr = orc.step_ions(net["mechs"], st0, net["v0"], n, 0.025)
    scale = np.zeros(n)
    for m, s in zip(net["mechs"], st0):
        c, _ = orc.mech_currents(m["type"], m["params"], m["node_index"], net["v0"], s)
        np.add.at(scale, m["node_index"], np.abs(c))
    assert np.all(np.abs(rhs.cpu().numpy() - rr) <= TOL_FP64 * (scale + 1e-300))
    assert np.max(np.abs(v.cpu().numpy() - vr) / np.maximum(np.abs(vr), 1.0)) <= 1e-11
    for q in (1, 2, 3):
        assert np.all(np.abs(ions[q - 1].cpu().numpy() - ir[q]) <= TOL_FP64 * (scale + 1e-300))
    for m, s in zip(ms, sr):
        got = m.states().cpu().numpy()
        if m.type == W.TYPE_CACUM:
            err = np.max(np.abs(got - s) / np.maximum(np.abs(s), 1e-12))
            assert err <= 1e-10, err
        else:
            assert state_err(got, s) <= 1e-11, (m.type, state_err(got, s))
    assert ctx.plan(ms)["fused"] == 1


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_network_fused_and_per_mechanism_paths_agree(api, orc, prec):
    """The ion-tagged network with the 3-state scheme and the buffer in the
    fused tile kernel (several tiles) against the per-mechanism launch
    sequence (forced by the no_fuse option): v, rhs, d,
    the ion arrays and every state after 12 steps."""
    net = W.cortical_ions(3000, seed=22)
    n = net["n_nodes"]
    P = api.NMODL_FP64 if prec == "fp64" else api.NMODL_MIXED
    res = {}
    for form in ("fused", "per_mechanism"):
        ctx = api.Context(0, precision=P, tile_smem=24 * 1024, window=5,
                          no_fuse=int(form == "per_mechanism"))
        ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
        ctx.set_ions(*ions)
        ms = [mech(api, ctx, m, n) for m in net["mechs"]]
        v = to_dev(net["v0"])
        for m in ms:
            m.init(v)
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
        d = torch.zeros_like(rhs)
        ctx.step(ms, 0.025, 1.0, v, rhs, d, 12)
        assert ctx.sync() == 0
        plan = ctx.plan(ms)
        assert plan["fused"] == (form == "fused")
        if form == "fused":
            assert plan["tiles"] > 1
        res[form] = (v.cpu().numpy(), rhs.cpu().numpy(), d.cpu().numpy(),
                     [x.cpu().numpy() for x in ions],
                     [m.states().cpu().numpy() for m in ms[:len(net["mechs"])]])
    (vf, rf, df, iof, sf), (vg, rg, dg, iog, sg) = res["fused"], res["per_mechanism"]
    if prec == "fp64":
        assert np.max(np.abs(vf - vg) / np.maximum(np.abs(vg), 1.0)) <= 1e-10
        assert np.max(np.abs(df - dg) / dg) <= 1e-11
        for a, b in zip(iof, iog):
            assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.abs(b).max())
        for a, b in zip(sf, sg):
            if a.size:
                assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3)) <= 1e-9
    else:
        assert np.max(np.abs(vf - vg)) <= 1e-3
        for a, b in zip(sf, sg):
            if a.size:
                assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3)) <= 1e-4
        # the ion currents (the fused MIXED form sums FP32 conductance
        # factors, the launches FP64 conductances of the same states)
        for a, b in zip(iof, iog):
            assert np.max(np.abs(a - b)) <= 1e-4 * max(1.0, np.abs(b).max())
    cai = sf[-1][0]
    assert np.all(np.isfinite(cai)) and cai.min() >= 0


def test_network_trajectory_and_determinism(api, orc):
    net = W.cortical_ions(1500, seed=18)
    n = net["n_nodes"]
    a = _run_network(api, net, 40)
    b = _run_network(api, net, 40)
    for x, y in zip(a[5], b[5]):
        assert torch.equal(x, y)
    assert torch.equal(a[2], b[2])
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], net["v0"])
           for m in net["mechs"]]
    vr, rr, dr, ir, sr = orc.step_ions(net["mechs"], st0, net["v0"], n, 0.025, nsteps=40)
    vg = a[2].cpu().numpy()
    ok = np.abs(vg - vr) <= 1e-9 * np.maximum(np.abs(vr), 1.0)
    assert ok.mean() >= 0.999, ok.mean()  # spike thresholds amplify 1-ulp exp differences
    cai = [m for m in a[1] if m.type == W.TYPE_CACUM][0].states().cpu().numpy()[0]
    assert np.all(np.isfinite(cai)) and cai.min() >= 0


def test_plan_forms(api):
    """Ion arrays keep the fused plan; the no_fuse option gives the
    per-mechanism plan and switching it back the fused one; unregistering
    the arrays keeps the fused plan."""
    net = W.cortical_mix(2000, seed=19)
    n = net["n_nodes"]
    ctx = api.Context(0)
    ms = [mech(api, ctx, m, n) for m in net["mechs"]]
    v = to_dev(net["v0"])
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    d = torch.zeros_like(rhs)
    ina = torch.zeros_like(rhs)
    ctx.set_ions(ina=ina)
    ctx.step(ms, 0.025, 1.0, v, rhs, d, 3)
    assert ctx.plan(ms)["fused"] == 1
    ctx.set_options(no_fuse=1)
    ctx.step(ms, 0.025, 1.0, v, rhs, d, 3)
    assert ctx.plan(ms)["fused"] == 0
    ctx.set_options(no_fuse=0)
    ctx.set_ions()
    ctx.step(ms, 0.025, 1.0, v, rhs, d, 3)
    assert ctx.plan(ms)["fused"] == 1
    assert ctx.sync() == 0


def test_fused_with_empty_small_systems(api, orc):
    """Empty 3-state and buffer mechanisms in a fused list change nothing."""
    net = W.cortical_mix(600, seed=24)
    n = net["n_nodes"]
    ctx = api.Context(0)
    ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    ctx.set_ions(*ions)
    ms = [mech(api, ctx, m, n) for m in net["mechs"]]
    empty = [api.Mechanism(ctx, api.NMODL_KIN3, np.zeros(0, np.int32), n,
                           W.kin3_params(W.Stream(1, 1))),
             api.Mechanism(ctx, api.NMODL_CACUM, np.zeros(0, np.int32), n, W.cacum_params())]
    v = to_dev(net["v0"])
    for m in ms:
        m.init(v)
    rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
    d = torch.zeros_like(rhs)
    ctx.step(ms + empty, 0.025, 1.0, v, rhs, d, 6)
    assert ctx.sync() == 0 and ctx.plan(ms + empty)["fused"] == 1
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], net["v0"])
           for m in net["mechs"]]
    v_ref, _, d_ref, _ = orc.step(net["mechs"], st0, net["v0"], n, 0.025, nsteps=6)
    assert np.max(np.abs(v.cpu().numpy() - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-10
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-11)


def test_cable_with_ions_fused_matches_per_step(api):
    """Cells of compartments with ion arrays, the 3-state scheme and the
    buffer: the fused cable form (tiles of whole cells, EXT kernel) against
    the per-step launch sequence of the same step (itself checked against the
    oracle by the cable and ion tests)."""
    cab = W.cable_cells(60, seed=25, size_lo=5, size_hi=80)
    n = cab["n_nodes"]
    net = W.cortical_ions(n, seed=25, kin3_frac=0.5)
    res = {}
    for form in ("fused", "per_step"):
        ctx = api.Context(0, tile_smem=48 * 1024, window=6, no_fuse=int(form == "per_step"))
        ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
        ctx.set_ions(*ions)
        ms = [mech(api, ctx, m, n) for m in net["mechs"]]
        v = to_dev(net["v0"])
        for m in ms:
            m.init(v)
        cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
        rhs = torch.zeros(n, dtype=torch.float64, device="cuda:0")
        d = torch.zeros_like(rhs)
        cable.step(ms, 0.025, 1.0, v, rhs, d, 15)
        assert ctx.sync() == 0
        assert ctx.plan(ms)["fused"] == (form == "fused")
        res[form] = (v.cpu().numpy(), d.cpu().numpy(), [x.cpu().numpy() for x in ions],
                     [m.states().cpu().numpy() for m in ms[:len(net["mechs"])]])
        cable.close()
    (vf, df, iof, sf), (vg, dg, iog, sg) = res["fused"], res["per_step"]
    assert np.max(np.abs(vf - vg) / np.maximum(np.abs(vg), 1.0)) <= 1e-10
    assert np.max(np.abs(df - dg) / dg) <= 1e-11
    for a, b in zip(iof, iog):
        assert np.max(np.abs(a - b)) <= 1e-10 * max(1.0, np.abs(b).max())
    for a, b in zip(sf, sg):
        if a.size:
            assert np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-3)) <= 1e-9
