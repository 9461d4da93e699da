"""Parity at the shapes the benchmark runs, with the plans it runs them in.

* Cable form: the benchmark's 10,000 cells of 20..400 compartments (tree
  morphologies) with the cortical channel mix, autotuned fused plan (tiles
  of whole cells, level-scheduled tree solve in shared memory), 200 steps.
  Checked on 1,000 whole cells that the oracle integrates as their own
  network (cells are not coupled to each other): the 20 largest cells (the
  largest tiles), the 10 deepest trees (the longest level schedules) and
  970 random cells of at most 100 compartments.  The oracle solves each
  cell's tree system by dense LU with partial pivoting, O(n^3) per cell and
  step, so its cells run in a pool of processes (started with spawn).
* Ion network: the benchmark's ion-tagged cortical mix on 2,000,000 nodes
  (10 cnexp types writing ina/ik/ica, a 3-state potassium scheme on half of
  the nodes, a calcium buffer on every node reading ica), fused plan, 200
  steps, checked on 1,500 sampled nodes.

Both at the trajectory tolerance 1e-9 (FP64); each side starts from its own
INITIAL.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import make_mechs, oracle_cable_cells, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

TOL = 1e-9


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _cells_subnet(wl, cab, cells):
    """The network of the given whole cells, renumbered (cells in order)."""
    off = cab["offsets"]
    nodes = np.concatenate([np.arange(off[c], off[c + 1]) for c in cells])
    remap = -np.ones(wl["n_nodes"], dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    mechs, sel = [], []
    for m in wl["mechs"]:
        keep = remap[m["node_index"]] >= 0
        sel.append(np.nonzero(keep)[0])
        mechs.append(dict(type=m["type"], params=m["params"],
                          node_index=remap[m["node_index"][keep]].astype(np.int32)))
    par = cab["parent"][nodes]
    par = np.where(par < 0, -1, remap[np.maximum(par, 0)]).astype(np.int32)
    return dict(nodes=nodes, n_nodes=nodes.size, mechs=mechs, parent=par,
                ga=cab["ga"][nodes], gb=cab["gb"][nodes], v0=wl["v0"][nodes]), sel


def test_cable_benchmark_network_sampled_parity(api, orc):
    cab = W.cable_cells(10000, seed=7)
    wl = W.cortical_mix(cab["n_nodes"], seed=2)
    n = cab["n_nodes"]
    ctx = api.Context(0)
    mechs = make_mechs(ctx, wl)
    v = to_dev(wl["v0"])
    for m in mechs:
        m.init(v)
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    cable.step(mechs, 0.025, 1.0, v, rhs, d, 200)
    assert ctx.sync() == 0
    plan = ctx.plan(mechs)
    assert plan["fused"]

    # the sample: largest cells, deepest trees, random small cells
    off = cab["offsets"]
    sizes = np.diff(off)
    depth = np.zeros(n, dtype=np.int64)
    par = cab["parent"]
    for i in range(n):
        if par[i] >= 0:
            depth[i] = depth[par[i]] + 1
    cell_depth = np.maximum.reduceat(depth, off[:-1])
    largest = np.argsort(-sizes, kind="stable")[:20]
    big = set(largest.tolist())
    deepest = [c for c in np.argsort(-cell_depth, kind="stable") if c not in big][:10]
    small = np.nonzero(sizes <= 100)[0]
    small = np.setdiff1d(small, np.concatenate([largest, deepest]))
    rnd = W.Stream(81, 1).integers(4000, 0, small.size - 1)
    pick = []
    for r in rnd:
        c = small[r]
        if c not in pick:
            pick.append(c)
        if len(pick) == 970:
            break
    cells = np.sort(np.concatenate([largest, deepest, np.array(pick)]).astype(np.int64))
    assert cells.size == 1000 and sizes[cells].max() == sizes.max()

    # oracle (built by the orc fixture before the pool starts): chunks of
    # cells balanced by their n^3 cost, one process each
    nproc = max(1, min(16, os.cpu_count() or 1))
    cost = sizes[cells].astype(np.float64) ** 3
    chunks = [[] for _ in range(nproc)]
    load = np.zeros(nproc)
    for c in cells[np.argsort(-cost, kind="stable")]:
        k = int(np.argmin(load))
        chunks[k].append(c)
        load[k] += float(sizes[c]) ** 3
    subs = [(_cells_subnet(wl, cab, np.sort(np.array(ch))) if ch else None) for ch in chunks]
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.starmap(oracle_cable_cells, [(s[0], 200) for s in subs if s is not None])
    vg, dg, rg = v.cpu().numpy(), d.cpu().numpy(), rhs.cpu().numpy()
    states = [m.states().cpu().numpy() if m.n_states else None for m in mechs]
    checked = 0
    for (sub, sel), (v_ref, r_ref, d_ref, s_ref) in zip([s for s in subs if s is not None], res):
        nodes = sub["nodes"]
        ev = np.max(np.abs(vg[nodes] - v_ref) / np.maximum(np.abs(v_ref), 1.0))
        assert ev <= TOL, ev
        np.testing.assert_allclose(dg[nodes], d_ref, rtol=TOL)
        assert np.max(np.abs(rg[nodes] - r_ref) / (200 * d_ref)) <= TOL
        for st, idx, s in zip(states, sel, s_ref):
            if st is not None:
                assert state_err(st[:, idx], s) <= TOL
        checked += nodes.size
    assert checked == int(sizes[cells].sum())
    cable.close()
    for m in mechs:
        m.close()
    ctx.close()


def test_ion_benchmark_network_sampled_parity(api, orc):
    wl = W.cortical_ions(2_000_000, seed=8)
    n = wl["n_nodes"]
    ctx = api.Context(0)
    ions = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    ctx.set_ions(*ions)
    mechs = [api.Mechanism(ctx, m["type"], m["node_index"], n, m["params"],
                           ion=m.get("ion", 0)) for m in wl["mechs"]]
    v = to_dev(wl["v0"])
    for m in mechs:
        m.init(v)
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, 200)
    assert ctx.sync() == 0
    assert ctx.plan(mechs)["fused"]

    nodes = np.unique(W.Stream(83, 1).integers(1600, 0, n - 1))[:1500]
    assert nodes.size == 1500
    remap = -np.ones(n, dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    sub, sel = [], []
    for m in wl["mechs"]:
        keep = remap[m["node_index"]] >= 0
        sel.append(np.nonzero(keep)[0])
        sub.append(dict(type=m["type"], params=m["params"], ion=m.get("ion", 0),
                        node_index=remap[m["node_index"][keep]].astype(np.int32)))
    v0 = wl["v0"][nodes]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], v0) for m in sub]
    v_ref, r_ref, d_ref, ion_ref, s_ref = orc.step_ions(sub, st0, v0, nodes.size, 0.025,
                                                        nsteps=200)
    vg = v.cpu().numpy()[nodes]
    assert np.max(np.abs(vg - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= TOL
    np.testing.assert_allclose(d.cpu().numpy()[nodes], d_ref, rtol=TOL)
    assert np.max(np.abs(rhs.cpu().numpy()[nodes] - r_ref) / (200 * d_ref)) <= TOL
    for k in range(3):
        got = ions[k].cpu().numpy()[nodes]
        ref = ion_ref[k + 1]
        # against the node's current scale: 200 mV x d
        assert np.max(np.abs(got - ref) / (200 * d_ref)) <= TOL, k
    for m, idx, s in zip(mechs, sel, s_ref):
        if m.n_states:
            st = m.states()[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy()
            assert state_err(st, s) <= TOL, m.type
    for m in mechs:
        m.close()
    ctx.close()
