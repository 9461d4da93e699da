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
