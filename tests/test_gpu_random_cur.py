"""Seeded random current updates (nmodl_cur) against the oracle.

Each case draws a mechanism kind (HH, a cnexp channel type, the 3-state or
9-state scheme), a node count and a sorted node_index whose per-node
multiplicities range from none to several hundred (runs shorter than,
equal to and longer than a warp, straddling 32-wide pieces), states from
the oracle's INITIAL at random voltages, and nonzero rhs and d to add to.
rhs and d after the update must match the oracle's per-node sums in
mechanism order: d to 1e-12 relative, rhs to 1e-12 of the node's summed
current magnitude; nodes without instances keep their values bit for bit."""
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


def _case(seed):
    s = W.Stream(seed, 3001)
    kind = int(s.integers(1, 0, 3)[0])
    n = int(s.integers(1, 1, 5000)[0])
    # multiplicities: mostly 0-3, a few long runs
    mult = s.integers(n, 0, 3)
    long_nodes = s.integers(int(s.integers(1, 0, 6)[0]), 0, n - 1)
    for k, nd in enumerate(long_nodes):
        mult[nd] = (31, 32, 33, 257, 500, 64)[k % 6]
    ni = np.repeat(np.arange(n), mult).astype(np.int32)
    if kind == 0:
        mt, p = W.TYPE_HH, W.hh_params()
    elif kind == 1:
        mt, p = W.TYPE_CNEXP, W.cortical_type_params(seed)[int(s.integers(1, 0, 9)[0])]
    elif kind == 2:
        mt, p = W.TYPE_KIN3, W.kin3_params(W.Stream(seed, 3002))
    else:
        mt, p = W.TYPE_KIN9, W.kin9_params(W.Stream(seed, 3003))
    v = s.uniform(n, -90.0, 40.0)
    rhs0 = s.uniform(n, -1.0, 1.0)
    d0 = s.uniform(n, 1.0, 2.0)
    return mt, p, ni, n, v, rhs0, d0


@pytest.mark.parametrize("seed", range(30))
def test_random_current_update_matches_the_oracle(api, orc, seed):
    mt, p, ni, n, v, rhs0, d0 = _case(seed)
    ctx = api.Context(0)
    m = api.Mechanism(ctx, mt, ni, n, p)
    st = orc.mech_init(mt, p, ni, v)
    if m.n_states:
        m.set_states(to_dev(st))
    rhs, d = to_dev(rhs0), to_dev(d0)
    m.cur(to_dev(v), rhs, d)
    assert ctx.sync() == 0
    r_ref, d_ref = orc.mech_cur(mt, p, ni, v, st, rhs0, d0)
    c, _ = orc.mech_currents(mt, p, ni, v, st)
    scale = np.zeros(n)
    np.add.at(scale, ni, np.abs(c))
    got_r, got_d = rhs.cpu().numpy(), d.cpu().numpy()
    assert np.all(np.abs(got_r - r_ref) <= 1e-12 * (scale + np.abs(rhs0))), seed
    np.testing.assert_allclose(got_d, d_ref, rtol=1e-12)
    empty = np.bincount(ni, minlength=n) == 0
    assert np.array_equal(got_r[empty], rhs0[empty]) and np.array_equal(got_d[empty], d0[empty])
    m.close()
    ctx.close()
