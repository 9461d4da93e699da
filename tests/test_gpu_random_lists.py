"""Seeded random mechanism lists through nmodl_step, FP64, against the oracle.

Each case draws a network (300-4,000 nodes) and a list from every mechanism
kind the step covers -- HH, a random subset of the ten cnexp channel types,
the 3-state and 9-state schemes, and, with ion arrays, the calcium buffer --
each on a random fraction of the nodes with one or two instances per chosen
node; with ion arrays the currents carry their ion tags.  The plan options
are drawn too (tile budget, block size, window; or left to the autotuner),
so that the planner meets lists, tile shapes and windows the hand-written
cases do not.  Whatever form the plan takes, v, d, the states and the ion
currents must match the oracle: FP64 one step at 1e-12, several windows at
1e-10; mixed precision (FP32 rates, FP64 accumulation) v within 1e-5 mV
after one step and 1e-4 mV after several, states within 1e-6 and 1e-5
absolute (the buffer's cai 1e-5 and 1e-4 relative), d 1e-6 relative."""
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


def _node_index(s, n, lo=0.1, hi=1.0):
    frac = float(s.uniform(1, lo, hi)[0])
    sel = np.nonzero(s.uniform(n) < frac)[0]
    k = s.integers(sel.size, 1, 2)  # one or two instances per chosen node
    return np.repeat(sel, k).astype(np.int32)


def _random_case(seed):
    s = W.Stream(seed, 1001)
    n = int(s.integers(1, 300, 4000)[0])
    ions = bool(s.integers(1, 0, 1)[0])
    mechs = []
    if s.uniform(1)[0] < 0.5:
        mechs.append(dict(type=W.TYPE_HH, params=W.hh_params(), node_index=_node_index(s, n),
                          name="hh"))
    blocks = W.cortical_type_params(seed)
    for (name, _, _), p in zip(W.CORTICAL_TYPES, blocks):
        if s.uniform(1)[0] < 0.6:
            m = dict(type=W.TYPE_CNEXP, params=p, node_index=_node_index(s, n), name=name)
            if ions:
                m["ion"] = W.CORTICAL_IONS[name]
            mechs.append(m)
    if s.uniform(1)[0] < 0.5:
        mechs.append(dict(type=W.TYPE_KIN3, params=W.kin3_params(W.Stream(seed, 1002)),
                          node_index=_node_index(s, n, 0.1, 0.6), name="kin3",
                          ion=W.ION_K if ions else 0))
    if s.uniform(1)[0] < 0.5:
        mechs.append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(seed, 1003)),
                          node_index=_node_index(s, n, 0.05, 0.4), name="kin9",
                          ion=W.ION_NA if ions else 0))
    if ions and s.uniform(1)[0] < 0.7:
        mechs.append(dict(type=W.TYPE_CACUM, params=W.cacum_params(),
                          node_index=np.arange(n, dtype=np.int32), name="cacum", ion=0))
    if not mechs:
        mechs.append(dict(type=W.TYPE_CNEXP, params=blocks[0], node_index=_node_index(s, n),
                          name="NaT"))
    opt = {}
    tile = int(s.integers(1, 0, 3)[0])
    if tile:
        opt["tile_smem"] = (16, 24, 48)[tile - 1] * 1024
    blk = int(s.integers(1, 0, 3)[0])
    if blk:
        opt["block"] = (128, 256, 512)[blk - 1]
    window = int(s.integers(1, 1, 4)[0])
    opt["window"] = window
    nsteps = window + int(s.integers(1, 0, 2 * window)[0])
    v0 = s.uniform(n, -90.0, 40.0)
    return dict(n_nodes=n, mechs=mechs, v0=v0), ions, opt, nsteps


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
@pytest.mark.parametrize("seed", range(40))
def test_random_list_matches_the_oracle(api, orc, seed, prec):
    wl, ions, opt, nsteps = _random_case(seed)
    n = wl["n_nodes"]
    mixed = prec == "mixed"
    if mixed:
        opt = dict(opt, precision=api.NMODL_MIXED)
    ctx = api.Context(0, **opt)
    arrs = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
    if ions:
        ctx.set_ions(*arrs)
    ms = [api.Mechanism(ctx, m["type"], m["node_index"], n, m["params"], ion=m.get("ion", 0))
          for m in wl["mechs"]]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"]) for m in wl["mechs"]]
    for m, x in zip(ms, st0):
        if m.n_states:
            m.set_states(to_dev(x))
    v = to_dev(wl["v0"])
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    for done in sorted({1, nsteps}):
        steps = 1 if done == 1 else nsteps - 1
        ctx.step(ms, 0.025, 1.0, v, rhs, d, steps)
        assert ctx.sync() == 0
        if ions:
            vr, rr, dr, ir, sr = orc.step_ions(wl["mechs"], st0, wl["v0"], n, 0.025, nsteps=done)
        else:
            vr, rr, dr, sr = orc.step(wl["mechs"], st0, wl["v0"], n, 0.025, nsteps=done)
        if mixed:
            v_tol, s_tol, c_tol, d_tol = (1e-5, 1e-6, 1e-5, 1e-6) if done == 1 else (1e-4, 1e-5, 1e-4, 1e-6)
            ev = np.max(np.abs(v.cpu().numpy() - vr))
        else:
            tol = TOL_FP64 if done == 1 else 1e-10
            v_tol, s_tol, c_tol, d_tol = tol, tol, max(1e-10, 10 * tol), tol
            ev = np.max(np.abs(v.cpu().numpy() - vr) / np.maximum(np.abs(vr), 1.0))
        assert ev <= v_tol, (seed, done, ev, ctx.plan(ms), opt)
        np.testing.assert_allclose(d.cpu().numpy(), dr, rtol=d_tol)
        for m, x in zip(ms, sr):
            if not m.n_states:
                continue
            got = m.states().cpu().numpy()
            if m.type == W.TYPE_CACUM:  # cai spans decades: relative to itself
                err = np.max(np.abs(got - x) / np.maximum(np.abs(x), 1e-12))
                assert err <= c_tol, (seed, done, m.type, err)
            else:
                err = np.max(np.abs(got - x)) if mixed else state_err(got, x)
                assert err <= s_tol, (seed, done, m.type, err)
        if ions and not mixed:
            # the ion currents of the last step, against the largest current
            for q in range(3):
                scale = max(np.abs(ir[q + 1]).max(), 1e-12)
                assert np.max(np.abs(arrs[q].cpu().numpy() - ir[q + 1])) <= 1e-9 * scale
    for m in ms:
        m.close()
    ctx.close()
