"""The 9-state kinetic scheme inside the fused tile kernel: networks that
mix cnexp channels with the 9-state scheme run all mechanism types in one
launch per window (the KIN variant of the tile kernel, one thread per
9-state instance running its banded Newton solve).  Checked against the
FP64 oracle (one step at 1e-12, a 45-step trajectory across several windows
at 1e-9), against the per-mechanism launch sequence of the same list, in
mixed precision, with ion arrays, and in the cable form; both builds of the
variant (blocks of at most 256 threads: the solve in registers; larger
blocks: the wide build, FP64 768 threads, MIXED 512, with part of the solve
in local memory)."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import TOL_FP64, node_scale, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _network(n_nodes, seed, frac=0.3, ions=False):
    """The cortical mix (or its ion-tagged form) with the 9-state scheme on
    a seeded fraction of the nodes (one instance each), last in the list."""
    wl = W.cortical_ions(n_nodes, seed=seed) if ions else W.cortical_mix(n_nodes, seed=seed)
    s = W.Stream(seed, 901)
    ni = np.nonzero(s.uniform(n_nodes) < frac)[0].astype(np.int32)
    wl["mechs"].append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(4, 401)),
                            node_index=ni, name="kin9", ion=W.ION_NA if ions else 0))
    return wl


def _run(api, orc, wl, steps, ions=False, **opt):
    n = wl["n_nodes"]
    ctx = api.Context(0, **opt)
    arrs = None
    if ions:
        arrs = [torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)]
        ctx.set_ions(*arrs)
    mechs = [api.Mechanism(ctx, m["type"], m["node_index"], n, m["params"],
                           ion=m.get("ion", 0)) for m in wl["mechs"]]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"]) for m in wl["mechs"]]
    for m, s in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(s))
    v = to_dev(wl["v0"])
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    ctx.step(mechs, 0.025, 1.0, v, rhs, d, steps)
    assert ctx.sync() == 0
    plan = ctx.plan(mechs)
    out = dict(v=v.cpu().numpy(), rhs=rhs.cpu().numpy(), d=d.cpu().numpy(),
               states=[m.states().cpu().numpy() if m.n_states else None for m in mechs],
               plan=plan, st0=st0, kin9_stats=mechs[-1].stats(),
               ions=[a.cpu().numpy() for a in arrs] if arrs else None)
    for m in mechs:
        m.close()
    ctx.close()
    return out


@pytest.mark.parametrize("block", [256, 768])
def test_fused_one_step_and_trajectory_fp64(api, orc, block):
    wl = _network(6000, seed=41)
    n = wl["n_nodes"]
    for steps, tol in ((1, TOL_FP64), (45, 1e-9)):
        got = _run(api, orc, wl, steps, tile_smem=24 * 1024, window=7, block=block)
        assert got["plan"]["fused"] and got["plan"]["tiles"] > 20
        assert got["plan"]["block"] == block
        v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], got["st0"], wl["v0"], n, 0.025,
                                              nsteps=steps)
        assert np.max(np.abs(got["v"] - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= tol
        if steps == 1:
            sr, sd = node_scale(orc, wl, got["st0"], wl["v0"])
            assert np.max(np.abs(got["rhs"] - r_ref) / (sr + 1e-300)) <= tol
            assert np.max(np.abs(got["d"] - d_ref) / (sd + 1e-3 / 0.025)) <= tol
        for g, s in zip(got["states"], s_ref):
            if g is not None:
                assert state_err(g, s) <= tol, steps


@pytest.mark.parametrize("block", [128, 512])
def test_fused_matches_the_per_mechanism_sequence(api, orc, block):
    wl = _network(3000, seed=42, frac=0.6)
    a = _run(api, orc, wl, 10, window=4, tile_smem=24 * 1024, block=block)  # fused (fixed tiles)
    b = _run(api, orc, wl, 10, window=4, no_fuse=1)
    assert a["plan"]["fused"] and not b["plan"]["fused"]
    assert np.max(np.abs(a["v"] - b["v"]) / np.maximum(np.abs(b["v"]), 1.0)) <= 1e-12
    np.testing.assert_allclose(a["d"], b["d"], rtol=1e-12)
    for x, y in zip(a["states"], b["states"]):
        if x is not None:
            assert state_err(x, y) <= 1e-12


@pytest.mark.parametrize("block", [256, 512])
def test_fused_mixed_precision(api, orc, block):
    wl = _network(4000, seed=43)
    n = wl["n_nodes"]
    got = _run(api, orc, wl, 20, precision=api.NMODL_MIXED, tile_smem=32 * 1024, block=block)
    assert got["plan"]["fused"] and got["plan"]["block"] == block
    v_ref, _, _, s_ref = orc.step(wl["mechs"], got["st0"], wl["v0"], n, 0.025, nsteps=20)
    assert np.max(np.abs(got["v"] - v_ref)) <= 1e-3
    for g, s in zip(got["states"], s_ref):
        if g is not None:
            assert np.max(np.abs(g - s)) <= 1e-5
    # the 9-state instances stay on the simplex
    k9 = got["states"][-1]
    assert np.max(np.abs(k9.sum(axis=0) - 1.0)) <= 1e-12


def test_fused_with_ion_arrays(api, orc):
    """The ion-tagged network (10 cnexp types, 3-state scheme, calcium
    buffer) with a sodium-tagged 9-state scheme: one fused step against the
    oracle's ion step, ion arrays included."""
    wl = _network(3000, seed=44, ions=True)
    n = wl["n_nodes"]
    got = _run(api, orc, wl, 1, ions=True, tile_smem=24 * 1024)
    assert got["plan"]["fused"]
    v_ref, r_ref, d_ref, ion_ref, s_ref = orc.step_ions(wl["mechs"], got["st0"], wl["v0"], n,
                                                        0.025, nsteps=1)
    assert np.max(np.abs(got["v"] - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= TOL_FP64
    for k in range(3):
        assert np.max(np.abs(got["ions"][k] - ion_ref[k + 1]) / (200 * d_ref)) <= TOL_FP64
    for g, s in zip(got["states"], s_ref):
        if g is not None:
            assert state_err(g, s) <= TOL_FP64


def test_fused_cable_form(api, orc):
    cab = W.cable_cells(30, seed=9, size_lo=5, size_hi=80)
    wl = W.cortical_mix(cab["n_nodes"], seed=45)
    s = W.Stream(45, 901)
    ni = np.nonzero(s.uniform(cab["n_nodes"]) < 0.4)[0].astype(np.int32)
    wl["mechs"].append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(4, 401)),
                            node_index=ni))
    n = cab["n_nodes"]
    ctx = api.Context(0, window=5)
    mechs = [api.Mechanism(ctx, m["type"], m["node_index"], n, m["params"]) for m in wl["mechs"]]
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"]) for m in wl["mechs"]]
    for m, x in zip(mechs, st0):
        if m.n_states:
            m.set_states(to_dev(x))
    cable = api.Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    cable.step(mechs, 0.025, 1.0, v, rhs, d, 12)
    assert ctx.sync() == 0
    assert ctx.plan(mechs)["fused"]
    v_ref, _, d_ref, s_ref = orc.step_cable(wl["mechs"], st0, wl["v0"], n, cab["parent"],
                                            cab["ga"], cab["gb"], 0.025, nsteps=12)
    assert np.max(np.abs(v.cpu().numpy() - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-10
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-12)
    for m, x in zip(mechs, s_ref):
        if m.n_states:
            assert state_err(m.states().cpu().numpy(), x) <= 1e-10
    cable.close()
    for m in mechs:
        m.close()
    ctx.close()


def test_autotuned_form_parity_and_counters(api, orc):
    """Default options (the autotuner may run an FP64 list with the 9-state
    scheme as per-mechanism launches where they time faster than the fused
    variant): whichever form it keeps, the trajectory matches the oracle, and
    the Newton counters equal those of an explicit per-mechanism run (the
    trial launches on scratch copies leave them untouched)."""
    wl = _network(20000, seed=46, frac=0.3)
    n = wl["n_nodes"]
    steps = 45
    got = _run(api, orc, wl, steps, window=9)
    ref_run = _run(api, orc, wl, steps, window=9, no_fuse=1)
    assert got["plan"]["form"] in ("tiles", "launches")
    v_ref, _, _, s_ref = orc.step(wl["mechs"], got["st0"], wl["v0"], n, 0.025, nsteps=steps)
    assert np.max(np.abs(got["v"] - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= 1e-9
    for g, s in zip(got["states"], s_ref):
        if g is not None:
            assert state_err(g, s) <= 1e-9
    assert got["kin9_stats"]["newton_iters"] == ref_run["kin9_stats"]["newton_iters"]
    assert got["kin9_stats"]["newton_iters"] >= 2 * steps * wl["mechs"][-1]["node_index"].size


@pytest.mark.parametrize("prec,block", [("fp64", 256), ("fp64", 768), ("mixed", 256), ("mixed", 512)])
def test_two_kinetic_mechanisms_share_the_first_work_group(api, orc, prec, block):
    """Two 9-state mechanisms (different rates, ragged counts: 0 to 2
    instances per node, 731 and 1,266 instances) beside the cnexp mix: their
    items form the one padded group at the head of the state phase's work
    order that the warps take in chunks.  One step against the FP64 oracle
    (FP64 at 1e-12; MIXED within the mixed form's state bound) and a 15-step
    window against the per-mechanism launches."""
    wl = _network(5003, seed=47, frac=0.15)
    s2 = W.Stream(48, 902)
    ni2 = np.sort(np.concatenate([np.nonzero(s2.uniform(5003) < 0.2)[0],
                                  np.nonzero(s2.uniform(5003) < 0.06)[0]])).astype(np.int32)
    wl["mechs"].append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(49, 401)),
                            node_index=ni2, name="kin9b"))
    n = wl["n_nodes"]
    opt = dict(tile_smem=24 * 1024, block=block)
    if prec == "mixed":
        opt["precision"] = api.NMODL_MIXED
    got = _run(api, orc, wl, 1, **opt)
    assert got["plan"]["fused"] and got["plan"]["block"] == block and got["plan"]["tiles"] > 10
    v_ref, _, _, s_ref = orc.step(wl["mechs"], got["st0"], wl["v0"], n, 0.025, nsteps=1)
    v_tol, s_tol = (TOL_FP64, TOL_FP64) if prec == "fp64" else (1e-4, 1e-5)
    assert np.max(np.abs(got["v"] - v_ref) / np.maximum(np.abs(v_ref), 1.0)) <= v_tol
    for g, s in zip(got["states"], s_ref):
        if g is not None:  # FP64 relative (state_err), MIXED absolute
            err = state_err(g, s) if prec == "fp64" else np.max(np.abs(g - s))
            assert err <= s_tol
    a = _run(api, orc, wl, 15, window=5, **opt)
    b_opt = {"precision": api.NMODL_MIXED} if prec == "mixed" else {}
    b = _run(api, orc, wl, 15, window=5, no_fuse=1, **b_opt)
    assert a["plan"]["fused"] and not b["plan"]["fused"]
    rt = 1e-12 if prec == "fp64" else 1e-4
    assert np.max(np.abs(a["v"] - b["v"]) / np.maximum(np.abs(b["v"]), 1.0)) <= rt
