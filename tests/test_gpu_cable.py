"""GPU parity of the cable step (per-cell tree solve replacing the diagonal
voltage update) against the FP64 oracle's dense per-cell solve."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import make_mechs, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _case(seed, n_cells):
    cab = W.cable_cells(n_cells, seed=seed, size_lo=3, size_hi=60)
    wl = W.cortical_mix(cab["n_nodes"], seed=seed + 20)
    return cab, wl


@pytest.mark.parametrize("use_graph,window", [(1, 40), (0, 3)])
def test_cable_step_fp64(api, orc, use_graph, window):
    cab, wl = _case(5, 40)
    n = cab["n_nodes"]
    ctx = api.Context(0, use_graph=use_graph, window=window)
    mechs = make_mechs(ctx, wl)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    for m, s in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(s))
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    assert cable.n_cells == 40
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cable.step(mechs, 0.025, 1.0, v, rhs, d, 10)
    assert ctx.sync() == 0
    v_ref, r_ref, d_ref, s_ref = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                                cab["ga"], cab["gb"], 0.025, nsteps=10)
    ev = np.max(np.abs(v.cpu().numpy() - v_ref) / np.maximum(np.abs(v_ref), 1.0))
    assert ev <= 1e-10, ev
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-12)
    assert np.max(np.abs(rhs.cpu().numpy() - r_ref) / (200 * d_ref)) <= 1e-10
    for m, s in zip(mechs, s_ref):
        if m.n_states:
            assert state_err(m.states().cpu().numpy(), s) <= 1e-10
    cable.close()


def test_cable_mixed_precision(api, orc):
    cab, wl = _case(6, 25)
    n = cab["n_nodes"]
    ctx = api.Context(0, precision=api.NMODL_MIXED)
    mechs = make_mechs(ctx, wl)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    for m, s in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(s))
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cable.step(mechs, 0.025, 1.0, v, rhs, d, 40)
    v_ref, _, _, s_ref = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                        cab["ga"], cab["gb"], 0.025, nsteps=40)
    assert np.max(np.abs(v.cpu().numpy() - v_ref)) <= 1e-3
    es = max(float(np.max(np.abs(m.states().cpu().numpy() - s)))
             for m, s in zip(mechs, s_ref) if m.n_states)
    assert es <= 1e-5
    cable.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_cable_fused_tiles_match_per_step_path(api, orc, prec):
    """The fused form (tiles of whole cells, tree solve in shared memory) on
    many small tiles against the oracle and against the per-step launch
    sequence (the no_fuse option): v, rhs, d, states."""
    cab, wl = _case(8, 120)
    n = cab["n_nodes"]
    P = api.NMODL_FP64 if prec == "fp64" else api.NMODL_MIXED
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    out = {}
    for form in ("fused", "per_step"):
        ctx = api.Context(0, precision=P, tile_smem=32 * 1024, window=7,
                          no_fuse=int(form == "per_step"))
        mechs = make_mechs(ctx, wl)
        for m, s in zip(mechs, st0):
            if m.n_states:
                m.set_states(to_dev(s))
        cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
        v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
        cable.step(mechs, 0.025, 1.0, v, rhs, d, 20)
        assert ctx.sync() == 0
        plan = ctx.plan(mechs)
        assert plan["fused"] == (form == "fused")
        if form == "fused":
            assert plan["tiles"] > 1
        out[form] = (v.cpu().numpy(), rhs.cpu().numpy(), d.cpu().numpy(),
                     [m.states().cpu().numpy() for m in mechs[:len(wl["mechs"])]])
        cable.close()
    v_ref, r_ref, d_ref, s_ref = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                                cab["ga"], cab["gb"], 0.025, nsteps=20)
    vf, rf, df, sf = out["fused"]
    if prec == "fp64":
        assert np.max(np.abs(vf - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-10
        np.testing.assert_allclose(df, d_ref, rtol=1e-12)
        assert np.max(np.abs(rf - r_ref) / (200 * d_ref)) <= 1e-10
        for a, b in zip(sf, s_ref):
            assert state_err(a, b) <= 1e-10
    else:
        assert np.max(np.abs(vf - v_ref)) <= 1e-3
        assert max(float(np.max(np.abs(a - b))) for a, b in zip(sf, s_ref) if a.size) <= 1e-5
    vg, rg, dg, _ = out["per_step"]
    tol = 1e-10 if prec == "fp64" else 1e-3
    assert np.max(np.abs(vf - vg)) <= tol * 100


def test_cable_clamped_holds_v(api, orc):
    cab, wl = _case(9, 30)
    n = cab["n_nodes"]
    ctx = api.Context(0, clamp_v=1)
    mechs = make_mechs(ctx, wl)
    v0 = to_dev(wl["v0"])
    for m in mechs:
        m.init(v0)
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    v, rhs, d = v0.clone(), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cable.step(mechs, 0.025, 1.0, v, rhs, d, 5)
    assert torch.equal(v, v0)
    # one step from the initial state: the assembled system against the oracle
    ctx2 = api.Context(0, clamp_v=1)
    mechs2 = make_mechs(ctx2, wl)
    for m in mechs2:
        m.init(v0)
    cable2 = api.Cable(ctx2, cab["parent"], cab["ga"], cab["gb"])
    cable2.step(mechs2, 0.025, 1.0, v, rhs, d, 1)
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
           for m in wl["mechs"]]
    _, r_ref, d_ref, _ = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                        cab["ga"], cab["gb"], 0.025, nsteps=1)
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-12)
    assert np.max(np.abs(rhs.cpu().numpy() - r_ref) / (200 * d_ref)) <= 1e-12
    assert ctx.sync() == 0 and ctx2.sync() == 0
    cable.close()
    cable2.close()


def test_cable_rejects_invalid_trees(api):
    ctx = api.Context(0)
    z = np.zeros(4)
    for parent in ([0, -1, 1, 2], [-1, 0, 3, 1], [-1, 0, -2, 2], [-1, 0, -1, 1]):
        with pytest.raises(api.NmodlError) as e:
            api.Cable(ctx, parent, z, z)
        assert e.value.status == -1
    api.Cable(ctx, [-1, 0, -1, 2], z, z).close()
