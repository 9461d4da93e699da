"""GPU parity of the 9-state kinetic scheme against the FP64 oracle:
stationary INITIAL, the implicit-Euler Newton step (FP64 and the FP32-LU +
FP64-refinement form), Newton counts, conservation, current, clamped step."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import TOL_FP64, make_mechs, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _setup(api, n, seed=4, **opts):
    wl = W.kin9_clamped(n, seed=seed)
    ctx = api.Context(0, **opts)
    (m,) = make_mechs(ctx, wl)
    return wl, ctx, m


def test_init_stationary(api, orc):
    wl, ctx, m = _setup(api, 3001)
    m.init(to_dev(wl["v0"]))
    spec = wl["mechs"][0]
    ref = orc.mech_init(spec["type"], spec["params"], spec["node_index"], wl["v0"])
    got = m.states().cpu().numpy()
    assert state_err(got, ref) <= 1e-11
    assert np.max(np.abs(got.sum(axis=0) - 1)) <= 1e-14
    assert ctx.sync() == 0


@pytest.mark.parametrize("dt", [0.025, 0.5])
def test_newton_step_fp64(api, orc, dt):
    wl, ctx, m = _setup(api, 4099)
    spec = wl["mechs"][0]
    m.set_states(to_dev(wl["x0"]))
    m.state(dt, to_dev(wl["v0"]))
    ref, iters = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                                wl["v0"], wl["x0"], dt, want_iters=True)
    got = m.states().cpu().numpy()
    assert state_err(got, ref) <= TOL_FP64, state_err(got, ref)
    st = m.stats()
    assert st["newton_iters"] == int(iters.sum())
    assert st["newton_max"] == int(iters.max())
    assert st["nonconverged"] == 0
    assert ctx.sync() == 0


def test_newton_trajectory_fp64(api, orc):
    wl, ctx, m = _setup(api, 2000)
    spec = wl["mechs"][0]
    v = to_dev(wl["v0"])
    m.set_states(to_dev(wl["x0"]))
    x = wl["x0"]
    for _ in range(200):
        m.state(0.025, v)
        x = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                           wl["v0"], x, 0.025)
    got = m.states().cpu().numpy()
    assert state_err(got, x) <= 1e-11
    assert np.max(np.abs(got.sum(axis=0) - 1)) <= 200 * 1e-15
    assert got.min() >= 0


def test_mixed_refinement(api, orc):
    """FP32 rates + FP32 LU, FP64 residual + refinement: error vs the FP64
    oracle (stated per quantity) and conservation to FP64 rounding."""
    wl, ctx, m = _setup(api, 4099, precision=api.NMODL_MIXED)
    spec = wl["mechs"][0]
    v = to_dev(wl["v0"])
    m.set_states(to_dev(wl["x0"]))
    m.state(0.025, v)
    ref = orc.mech_state(spec["type"], spec["params"], spec["node_index"],
                         wl["v0"], wl["x0"], 0.025)
    got = m.states().cpu().numpy()
    e1 = float(np.max(np.abs(got - ref)))
    cons = float(np.max(np.abs(got.sum(axis=0) - 1)))
    st = m.stats()
    print(f"KIN9 MIXED one-step abs err {e1:.2e}, |sum-1| {cons:.2e}, "
          f"mean updates {st['newton_iters'] / 4099:.2f}, max {st['newton_max']}")
    assert e1 <= 1e-6
    assert cons <= 1e-14
    assert st["nonconverged"] == 0
    assert ctx.sync() == 0


def test_cur_and_clamped_step(api, orc):
    wl, ctx, m = _setup(api, 1501, clamp_v=1)
    spec = wl["mechs"][0]
    m.set_states(to_dev(wl["x0"]))
    n = wl["n_nodes"]
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx.step([m], 0.025, 1.0, v, rhs, d, 7)
    assert ctx.sync() == 0
    v_ref, r_ref, d_ref, s_ref = orc.step(wl["mechs"], [wl["x0"]], wl["v0"], n, 0.025,
                                          nsteps=7, clamp_v=True)
    assert torch.equal(v, to_dev(wl["v0"]))
    assert state_err(m.states().cpu().numpy(), s_ref[0]) <= 1e-11
    np.testing.assert_allclose(d.cpu().numpy(), d_ref, rtol=1e-12)
    np.testing.assert_allclose(rhs.cpu().numpy(), r_ref, rtol=1e-11, atol=1e-15)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_kinetic_full_size_sampled_parity(api, orc, prec):
    """The kinetic benchmark's configuration: 1,000,000 clamped instances, 200
    clamped network steps (the per-mechanism launch sequence in graph
    windows), checked on 1,000 sampled instances against the oracle's own
    200-step trajectories (FP64 at the trajectory tolerance; MIXED, whose FP32
    rates change the solved system at ~1e-7 per step, within 2e-5)."""
    n = 1_000_000
    wl = W.kin9_clamped(n, seed=4)
    P = api.NMODL_FP64 if prec == "fp64" else api.NMODL_MIXED
    ctx = api.Context(0, precision=P, clamp_v=1)
    (m,) = make_mechs(ctx, wl)
    v = to_dev(wl["v0"])
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    m.set_states(to_dev(wl["x0"]))
    ctx.step([m], 0.025, 1.0, v, rhs, d, 200)
    assert ctx.sync() == 0
    idx = np.unique(W.Stream(78, 1).integers(1000, 0, n - 1))
    spec = wl["mechs"][0]
    sub_ni = np.arange(idx.size, dtype=np.int32)
    x = wl["x0"][:, idx]
    for _ in range(200):
        x = orc.mech_state(spec["type"], spec["params"], sub_ni, wl["v0"][idx], x, 0.025)
    got = m.states()[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy()
    if prec == "fp64":
        assert state_err(got, x) <= 1e-11, state_err(got, x)
    else:
        assert float(np.max(np.abs(got - x))) <= 2e-5, float(np.max(np.abs(got - x)))
    assert m.stats()["nonconverged"] == 0

