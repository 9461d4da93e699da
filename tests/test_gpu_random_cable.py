"""Seeded random cells and mechanism lists through the cable step, against the
oracle's per-cell solve.

Each case draws cells (1-12 cells of 1-400 compartments, branching with a
random probability, so that chains, bushy trees and single-compartment
cells all occur), a list of cnexp channel types (and sometimes HH and the
9-state scheme) on random fractions of the compartments, and the plan's
options (tile budget, block size, window, or the autotuner's choice).  FP64
after several windows: v and the states within 1e-10, d within 1e-12; MIXED
v within 1e-3 mV and the states within 1e-5."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _random_cable_case(seed):
    s = W.Stream(seed, 2001)
    n_cells = int(s.integers(1, 1, 12)[0])
    hi = int(s.integers(1, 1, 400)[0])
    cab = W.cable_cells(n_cells, seed=seed + 100, size_lo=1, size_hi=hi,
                        branch_p=float(s.uniform(1, 0.0, 0.6)[0]))
    n = cab["n_nodes"]
    mechs = []
    blocks = W.cortical_type_params(seed)
    for (name, _, _), p in zip(W.CORTICAL_TYPES, blocks):
        if s.uniform(1)[0] < 0.6:
            frac = float(s.uniform(1, 0.1, 1.0)[0])
            sel = np.nonzero(s.uniform(n) < frac)[0]
            k = s.integers(sel.size, 1, 2)
            mechs.append(dict(type=W.TYPE_CNEXP, params=p, node_index=np.repeat(sel, k).astype(np.int32),
                              name=name))
    if s.uniform(1)[0] < 0.3:
        sel = np.nonzero(s.uniform(n) < 0.5)[0].astype(np.int32)
        mechs.append(dict(type=W.TYPE_HH, params=W.hh_params(), node_index=sel, name="hh"))
    if s.uniform(1)[0] < 0.3:
        sel = np.nonzero(s.uniform(n) < 0.3)[0].astype(np.int32)
        mechs.append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(seed, 2002)),
                          node_index=sel, name="kin9"))
    if not mechs:
        mechs.append(dict(type=W.TYPE_CNEXP, params=blocks[9],
                          node_index=np.arange(n, dtype=np.int32), name="leak"))
    opt = {}
    tile = int(s.integers(1, 0, 2)[0])
    if tile:
        opt["tile_smem"] = (64, 104)[tile - 1] * 1024
    blk = int(s.integers(1, 0, 2)[0])
    if blk:
        opt["block"] = (256, 512)[blk - 1]
    window = int(s.integers(1, 1, 5)[0])
    opt["window"] = window
    nsteps = window + int(s.integers(1, 0, 2 * window)[0])
    v0 = s.uniform(n, -90.0, 40.0)
    return cab, dict(n_nodes=n, mechs=mechs, v0=v0), opt, nsteps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", range(20))
def test_random_cells_match_the_oracle(api, orc, seed, prec):
    cab, wl, opt, nsteps = _random_cable_case(seed)
    n = wl["n_nodes"]
    mixed = prec == "mixed"
    if mixed:
        opt = dict(opt, precision=api.NMODL_MIXED)
    ctx = api.Context(0, **opt)
    ms = [api.Mechanism(ctx, m["type"], m["node_index"], n, m["params"]) for m in wl["mechs"]]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"]) for m in wl["mechs"]]
    for m, x in zip(ms, st0):
        if m.n_states:
            m.set_states(to_dev(x))
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cable.step(ms, 0.025, 1.0, v, rhs, d, nsteps)
    assert ctx.sync() == 0
    v_ref, _, d_ref, s_ref = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                            cab["ga"], cab["gb"], 0.025, nsteps=nsteps)
    if mixed:
        assert np.max(np.abs(v.cpu().numpy() - v_ref)) <= 1e-3, (seed, opt)
        for m, x in zip(ms, s_ref):
            if m.n_states:
                assert np.max(np.abs(m.states().cpu().numpy() - x)) <= 1e-5, (seed, m.type)
    else:
        ev = np.max(np.abs(v.cpu().numpy() - v_ref) / np.maximum(np.abs(v_ref), 1.0))
        assert ev <= 1e-10, (seed, ev, opt, ctx.plan(ms))
        np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-12)
        for m, x in zip(ms, s_ref):
            if m.n_states:
                assert state_err(m.states().cpu().numpy(), x) <= 1e-10, (seed, m.type)
    cable.close()
    for m in ms:
        m.close()
    ctx.close()
