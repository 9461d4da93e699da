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


def test_cable_rejects_invalid_trees(api):
    ctx = api.Context(0)
    z = np.zeros(4)
    for parent in ([0, -1, 1, 2], [-1, 0, 3, 1], [-1, 0, -2, 2], [-1, 0, -1, 1]):
        with pytest.raises(api.NmodlError) as e:
            api.Cable(ctx, parent, z, z)
        assert e.value.status == -1
    api.Cable(ctx, [-1, 0, -1, 2], z, z).close()
