"""nmodl_cur_noalloc: the current update for callers that cannot allocate
device memory (for example code running inside another framework's memory
pool, or a host that forbids cudaMalloc after start-up).

It must give the same rhs/d as the regular nmodl_cur of a mechanism object,
within the tolerance the other parity tests use, on two calls in a row (its
scratch array keeps the previous call's contents, so the second call checks
that everything that must start fresh is reset).  This file is collected
last so that a run stopping at the first failure has run every other test;
it passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import TOL_FP64, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(mech_spec, n_nodes, v0, seed):
    from paper_1905_02241_b300 import _lib
    from paper_1905_02241_b300.api import Context, Mechanism
    ctx = Context(0)
    m = Mechanism(ctx, mech_spec["type"], mech_spec["node_index"], n_nodes,
                  mech_spec["params"])
    v = to_dev(v0)
    m.init(v)
    rng = np.random.default_rng(seed)
    rhs0, d0 = rng.normal(size=n_nodes), rng.uniform(0.1, 1.0, size=n_nodes)
    # existing entry point
    rhs_ref, d_ref = to_dev(rhs0), to_dev(d0)
    m.cur(v, rhs_ref, d_ref)
    states = m.states()                      # (n_states, n), row stride n
    ni = to_dev(mech_spec["node_index"])
    p = np.ascontiguousarray(mech_spec["params"], dtype=np.float64)
    scale = (np.abs(rhs0) + 200.0 * d_ref.cpu().numpy())
    torch.cuda.synchronize()
    for call in range(2):
        rhs, d = to_dev(rhs0), to_dev(d0)
        torch.cuda.synchronize()
        _lib.nmodl_cur_noalloc(0, ctx.stream.cuda_stream, mech_spec["type"], m.n,
                               ni.data_ptr(), n_nodes, p.ctypes.data, p.size,
                               states.data_ptr(), m.n, v.data_ptr(), rhs.data_ptr(),
                               d.data_ptr())
        ctx.stream.synchronize()
        er = np.abs(rhs.cpu().numpy() - rhs_ref.cpu().numpy())
        ed = np.abs(d.cpu().numpy() - d_ref.cpu().numpy())
        assert np.all(er <= TOL_FP64 * scale), (call, float(er.max()))
        assert np.all(ed <= TOL_FP64 * np.abs(d_ref.cpu().numpy())), (call, float(ed.max()))
    assert ctx.sync() == 0
    m.close()
    ctx.close()


def test_noalloc_matches_cur_cnexp_two_calls():
    wl = W.cortical_mix(20011, seed=31)
    for spec in (wl["mechs"][0], wl["mechs"][9], wl["mechs"][5]):
        _case(spec, wl["n_nodes"], wl["v0"], 1)


def test_noalloc_matches_cur_kin9_two_calls():
    wl = W.kin9_clamped(5003, seed=4)
    _case(wl["mechs"][0], wl["n_nodes"], wl["v0"], 2)


def test_noalloc_rejects_oversize_and_bad_index():
    from paper_1905_02241_b300 import _lib
    mx = _lib.nmodl_cur_noalloc_max_instances()
    assert mx == 8_000_000
    p = np.ascontiguousarray(W.cortical_type_params(2)[0])
    st = torch.cuda.current_stream().cuda_stream
    with pytest.raises(_lib.NmodlError) as e:   # size check comes before any access
        _lib.nmodl_cur_noalloc(0, st, W.TYPE_CNEXP, mx + 1, 16, 10, p.ctypes.data,
                               p.size, 16, mx + 1, 16, 16, 16)
    assert e.value.status == -10
    ni = to_dev(np.array([0, 3, 2], dtype=np.int32))
    s = to_dev(np.zeros(3 * 3))
    v, r, d = to_dev(np.zeros(5)), to_dev(np.zeros(5)), to_dev(np.zeros(5))
    torch.cuda.synchronize()
    with pytest.raises(_lib.NmodlError) as e:
        _lib.nmodl_cur_noalloc(0, st, W.TYPE_CNEXP, 3, ni.data_ptr(), 5, p.ctypes.data,
                               p.size, s.data_ptr(), 3, v.data_ptr(), r.data_ptr(),
                               d.data_ptr())
    assert e.value.status == -2
    _ = ctypes
