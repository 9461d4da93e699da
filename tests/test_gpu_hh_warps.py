"""The single-HH gate-warp step (one HH mechanism with one instance on each
node of a network of at most 32 nodes per SM: three warps per block, one
per gate, the current computed by each warp from the exchanged factors).
Checked against the FP64 oracle for one step (1e-12: v, rhs, d, states) and
over windows, against the per-mechanism launch sequence of the same list,
on ragged and degenerate sizes, clamped, and for the rules that keep other
lists on the tile kernel."""
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


def _wl(n, seed, lo=-100.0, hi=60.0):
    wl = W.hh_single(n, seed)
    wl["v0"] = W.Stream(seed, 9).uniform(n, lo, hi)
    return wl


def _run(api, orc, wl, nsteps, ions=False, **opt):
    n = wl["n_nodes"]
    ctx = api.Context(0, **opt)
    if ions:
        ctx.set_ions(*[torch.zeros(n, dtype=torch.float64, device="cuda:0") for _ in range(3)])
    spec = wl["mechs"][0]
    m = api.Mechanism(ctx, spec["type"], spec["node_index"], n, spec["params"])
    st0 = orc.mech_init(spec["type"], spec["params"], spec["node_index"], wl["v0"])
    m.set_states(to_dev(st0))
    v = to_dev(wl["v0"])
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    ctx.step([m], 0.025, 1.0, v, rhs, d, nsteps)
    assert ctx.sync() == 0
    out = dict(plan=ctx.plan([m]), st0=st0, v=v.cpu().numpy(), rhs=rhs.cpu().numpy(),
               d=d.cpu().numpy(), states=m.states().cpu().numpy())
    m.close()
    ctx.close()
    return out


def _check(orc, wl, got, nsteps, tol, clamp_v=0):
    n = wl["n_nodes"]
    v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], [got["st0"]], wl["v0"], n, 0.025,
                                          nsteps=nsteps, clamp_v=clamp_v)
    ev = np.max(np.abs(got["v"] - v_ref) / np.maximum(np.abs(v_ref), 1.0))
    es = state_err(got["states"], s_ref[0])
    ed = np.max(np.abs(got["d"] - d_ref) / np.abs(d_ref))
    if nsteps == 1:
        sr, _ = node_scale(orc, wl, [got["st0"]], wl["v0"])
        er = np.max(np.abs(got["rhs"] - r_ref) / (sr + 1e-300))
    else:  # the last step's terms at its own v: the cancellation-safe d * 200 mV
        er = np.max(np.abs(got["rhs"] - r_ref) / (200.0 * d_ref))
    assert ev <= tol and es <= tol and ed <= tol and er <= tol, (ev, es, ed, er)


@pytest.mark.parametrize("n", [4099, 4736, 1000, 37, 1])
def test_one_step_fp64(api, orc, n):
    """One step at 1e-12; 4099 nodes give 28 per block and a last block of
    11, 4736 = 32 per SM fills every block, 37 and 1 leave most lanes
    idle."""
    wl = _wl(n, seed=n)
    got = _run(api, orc, wl, 1)
    assert got["plan"]["form"] == "hh_gate_warps", got["plan"]
    _check(orc, wl, got, 1, TOL_FP64)


@pytest.mark.parametrize("steps,window", [(45, 7), (40, 40), (2, 1), (3, 2)])
def test_windows_fp64(api, orc, steps, window):
    wl = _wl(3001, seed=3)
    got = _run(api, orc, wl, steps, window=window)
    assert got["plan"]["form"] == "hh_gate_warps"
    _check(orc, wl, got, steps, 1e-10)


def test_clamped(api, orc):
    wl = _wl(2000, seed=4)
    got = _run(api, orc, wl, 12, clamp_v=1, window=5)
    assert got["plan"]["form"] == "hh_gate_warps"
    assert np.array_equal(got["v"], wl["v0"])
    _check(orc, wl, got, 12, 1e-11, clamp_v=1)


def test_matches_per_mechanism_launches(api, orc):
    wl = _wl(4096, seed=5, lo=-70.0, hi=-60.0)
    a = _run(api, orc, wl, 30, window=9)
    b = _run(api, orc, wl, 30, window=9, no_fuse=1)
    assert a["plan"]["form"] == "hh_gate_warps" and b["plan"]["form"] == "launches"
    assert np.max(np.abs(a["v"] - b["v"]) / np.maximum(np.abs(b["v"]), 1.0)) <= 1e-12
    assert state_err(a["states"], b["states"]) <= 1e-12
    np.testing.assert_allclose(a["d"], b["d"], rtol=1e-13)


def test_other_lists_keep_the_tile_kernel(api, orc):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # more than 32 nodes per SM
    wl = _wl(32 * sms + 1, seed=6)
    assert _run(api, orc, wl, 1)["plan"]["form"] == "tiles"
    # mixed precision, the Pade factor, ion arrays
    wl = _wl(1000, seed=7)
    assert _run(api, orc, wl, 1, precision=api.NMODL_MIXED)["plan"]["form"] == "tiles"
    assert _run(api, orc, wl, 1, cnexp_pade=1)["plan"]["form"] == "tiles"
    got = _run(api, orc, wl, 1, ions=True)
    assert got["plan"]["form"] == "tiles"
    _check(orc, wl, got, 1, TOL_FP64)
    # one instance on every node but not node i on instance i: a node with
    # two instances and one with none
    wl = _wl(1000, seed=8)
    ni = np.arange(1000, dtype=np.int32)
    ni[500] = 499
    wl["mechs"][0]["node_index"] = ni
    got = _run(api, orc, wl, 3)
    assert got["plan"]["form"] == "tiles"
    _check(orc, wl, got, 3, 1e-11)
