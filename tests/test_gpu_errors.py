"""Error paths of the C ABI on the device (no GPU fault is provoked: every
case is caught by argument checks, the index validation kernel, or the
non-finite latch that nmodl_sync reports)."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def api():
    from paper_1905_02241_b300 import api as A
    return A


def _create(api, ni, n_nodes=10, params=None, mtype=W.TYPE_CNEXP):
    ctx = api.Context(0)
    p = W.cortical_type_params(2)[0] if params is None else params
    return ctx, api.Mechanism(ctx, mtype, np.asarray(ni, np.int32), n_nodes, p)


def test_unsorted_index(api):
    with pytest.raises(api.NmodlError) as e:
        _create(api, [0, 2, 1])
    assert e.value.status == -2


def test_index_out_of_range(api):
    for ni in ([0, 1, 10], [-1, 0]):
        with pytest.raises(api.NmodlError) as e:
            _create(api, ni)
        assert e.value.status == -8


def test_bad_params(api):
    p = W.cortical_type_params(2)[0].copy()
    p[0] = 4  # too many gates
    with pytest.raises(api.NmodlError) as e:
        _create(api, [0, 1], params=p)
    assert e.value.status == -1
    with pytest.raises(api.NmodlError):
        _create(api, [0, 1], params=np.zeros(5))
    with pytest.raises(api.NmodlError):
        _create(api, [0, 1], params=W.hh_params(), mtype=99)


def test_bad_step_args(api):
    ctx, m = _create(api, [0, 1, 1])
    v, rhs, d = (to_dev(np.zeros(10)) for _ in range(3))
    with pytest.raises(api.NmodlError):
        ctx.step([m], -0.025, 1.0, v, rhs, d, 1)
    with pytest.raises(api.NmodlError):
        m.state(float("nan"), v)


def test_nonfinite_latched(api):
    ctx, m = _create(api, [0, 1, 1, 5])
    v = to_dev(np.full(10, -65.0))
    m.init(v)
    v[1] = float("nan")
    m.state(0.025, v)
    assert ctx.sync() == -5
    assert ctx.sync() == 0  # cleared after being reported


def test_nonfinite_node_sums_of_the_mixed_step_latched(api):
    # mixed precision forms a cnexp current's gbar m^p h^q in FP32: a gbar
    # beyond the FP32 range makes the node's conductance sums non-finite
    # while every state stays finite; the fused step must still report it
    n = 600
    ni = np.arange(n, dtype=np.int32)
    for ions in (False, True):
        ctx = api.Context(0, precision=api.NMODL_MIXED)
        if ions:
            ctx.set_ions(*[to_dev(np.zeros(n)) for _ in range(3)])
        big = W.cortical_type_params(3)[1].copy()
        big[1] = 1e300
        ms = [api.Mechanism(ctx, W.TYPE_CNEXP, ni, n, W.cortical_type_params(3)[0]),
              api.Mechanism(ctx, W.TYPE_CNEXP, ni[::7].copy(), n, big)]
        v = to_dev(np.full(n, -65.0))
        rhs, d = to_dev(np.zeros(n)), to_dev(np.zeros(n))
        for m in ms:
            m.init(v)
        ctx.step(ms, 0.025, 1.0, v, rhs, d, 3)
        assert ctx.plan(ms)["fused"]
        assert ctx.sync() == -5, ions
        got = v.cpu().numpy()
        assert not np.all(np.isfinite(got[::7])) and np.all(np.isfinite(np.delete(got, np.s_[::7])))
        for m in ms:
            m.close()
        ctx.close()


# -------------------------------------------- Newton non-convergence
# Provoked from the host with an iteration cap that no solve can meet (one
# update, then the convergence check never runs): every instance reports
# non-convergence, the context latches NMODL_ERR_NOCONV, nmodl_sync returns
# it once, and the same context then runs normally with the default cap.

def test_kinetic_nonconvergence_latched_and_counted(api):
    for prec in (api.NMODL_FP64, api.NMODL_MIXED):
        wl = W.kin9_clamped(1000, seed=4)
        ctx = api.Context(0, precision=prec, newton_max_iter=1, ir_max=0, clamp_v=1)
        (spec,) = wl["mechs"]
        m = api.Mechanism(ctx, spec["type"], spec["node_index"], wl["n_nodes"], spec["params"])
        m.set_states(to_dev(wl["x0"]))
        v = to_dev(wl["v0"])
        m.state(0.025, v)
        assert ctx.sync() == -6
        assert ctx.sync() == 0
        st = m.stats()
        assert st["nonconverged"] == 1000 and st["newton_max"] == 1
        ctx.set_options(newton_max_iter=8, ir_max=4)
        m.state(0.025, v)
        assert ctx.sync() == 0
        assert m.stats()["nonconverged"] == 1000
        m.close()
        ctx.close()


def test_buffer_nonconvergence_latched_standalone_and_fused(api):
    n = 2000
    ica = -to_dev(W.Stream(21, 2).loguniform(n, 1e-3, 1.0))
    v = to_dev(np.full(n, -65.0))
    for prec in (api.NMODL_FP64, api.NMODL_MIXED):
        ctx = api.Context(0, precision=prec, newton_max_iter=1, ir_max=0)
        ctx.set_ions(ica=ica)
        buf = api.Mechanism(ctx, W.TYPE_CACUM, np.arange(n, dtype=np.int32), n,
                            W.cacum_params())
        buf.init(v)
        buf.state(0.025, v)
        assert ctx.sync() == -6
        assert buf.stats()["nonconverged"] == n
        buf.close()
        ctx.close()
    # the fused tile kernel (the ion network's buffer items)
    wl = W.cortical_ions(3000, seed=8)
    ctx = api.Context(0, newton_max_iter=1)
    arrs = [to_dev(np.zeros(wl["n_nodes"])) for _ in range(3)]
    ctx.set_ions(*arrs)
    mechs = [api.Mechanism(ctx, m["type"], m["node_index"], wl["n_nodes"], m["params"],
                           ion=m.get("ion", 0)) for m in wl["mechs"]]
    vv = to_dev(wl["v0"])
    rhs, d = to_dev(np.zeros(wl["n_nodes"])), to_dev(np.zeros(wl["n_nodes"]))
    for m in mechs:
        m.init(vv)
    ctx.step(mechs, 0.025, 1.0, vv, rhs, d, 3)
    assert ctx.plan(mechs)["fused"]
    assert ctx.sync() == -6
    ctx.set_options(newton_max_iter=8)
    ctx.step(mechs, 0.025, 1.0, vv, rhs, d, 3)
    assert ctx.sync() == 0
    for m in mechs:
        m.close()
    ctx.close()


# -------------------------------------------------- bounded waits
# The tensor-core kernels wait on mbarriers with a poll limit.  The probe
# runs that wait on a barrier nothing arrives at: the limit runs out, the
# context latches NMODL_ERR_TIMEOUT, and the context stays usable.

def test_bounded_wait_timeout_latched_and_context_usable(api):
    from paper_1905_02241_b300 import _lib
    ctx, m = _create(api, [0, 1, 1, 5])
    v = to_dev(np.full(10, -65.0))
    m.init(v)
    assert ctx.sync() == 0
    _lib.nmodl_probe_wait(ctx.handle, 2000)
    assert ctx.sync() == -7
    assert ctx.sync() == 0
    m.state(0.025, v)
    assert ctx.sync() == 0
    with pytest.raises(api.NmodlError):
        _lib.nmodl_probe_wait(ctx.handle, 0)
    m.close()
    ctx.close()
