"""nmodl_cur_noalloc: the current update for callers that cannot allocate
device memory (for example code running inside another framework's memory
pool, or a host that forbids cudaMalloc after start-up).

On the same seeded inputs it must give the rhs/d of the FP64 CPU oracle and
of the regular nmodl_cur of a mechanism object, within the tolerance the
other parity tests use, on two calls in a row (its scratch array keeps the
previous call's contents, so the second call checks that everything that
must start fresh is reset).  The states it reads come from the oracle's own
INITIAL at one voltage and are evaluated at another, so they are not at
their steady state.  This file is collected last so that a run stopping at
the first failure has run every other test; it passes alone in a fresh
process as well as after the other tests.
"""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import TOL_FP64, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _case(orc, spec, n_nodes, v0, seed):
    from paper_1905_02241_b300 import _lib
    from paper_1905_02241_b300.api import Context, Mechanism
    rng = np.random.default_rng(seed)
    mtype, params, ni_h = spec["type"], spec["params"], spec["node_index"]
    st0 = orc.mech_init(mtype, params, ni_h, v0)
    v1 = v0 + rng.uniform(-15.0, 15.0, size=n_nodes)
    rhs0, d0 = rng.normal(size=n_nodes), rng.uniform(0.1, 1.0, size=n_nodes)
    r_orc, d_orc = orc.mech_cur(mtype, params, ni_h, v1, st0, rhs0, d0)
    c, g = orc.mech_currents(mtype, params, ni_h, v1, st0)
    scale_r, scale_d = np.abs(rhs0).copy(), np.abs(d0).copy()
    np.add.at(scale_r, ni_h, np.abs(c))
    np.add.at(scale_d, ni_h, np.abs(g))

    ctx = Context(0)
    m = Mechanism(ctx, mtype, ni_h, n_nodes, params)
    n = m.n
    states = to_dev(st0.reshape(-1, n) if st0.size else np.zeros((1, max(n, 1))))
    if m.n_states:
        m.set_states(states)
    v = to_dev(v1)
    rhs_ref, d_ref = to_dev(rhs0), to_dev(d0)
    m.cur(v, rhs_ref, d_ref)                  # the existing entry point
    assert ctx.sync() == 0
    rhs_ref, d_ref = rhs_ref.cpu().numpy(), d_ref.cpu().numpy()
    ni = to_dev(ni_h)
    p = np.ascontiguousarray(params, dtype=np.float64)
    torch.cuda.synchronize()
    for call in range(2):
        rhs, d = to_dev(rhs0), to_dev(d0)
        torch.cuda.synchronize()
        _lib.nmodl_cur_noalloc(0, ctx.stream.cuda_stream, mtype, n, ni.data_ptr(), n_nodes,
                               p.ctypes.data, p.size, states.data_ptr(), n, v.data_ptr(),
                               rhs.data_ptr(), d.data_ptr())
        ctx.stream.synchronize()
        r_h, d_h = rhs.cpu().numpy(), d.cpu().numpy()
        for want, name in ((r_orc, "oracle"), (rhs_ref, "nmodl_cur")):
            er = np.abs(r_h - want)
            assert np.all(er <= TOL_FP64 * scale_r), (call, name, float(er.max()))
        for want, name in ((d_orc, "oracle"), (d_ref, "nmodl_cur")):
            ed = np.abs(d_h - want)
            assert np.all(ed <= TOL_FP64 * scale_d), (call, name, float(ed.max()))
    m.close()
    ctx.close()


def test_noalloc_matches_oracle_and_cur_hh_two_calls(orc):
    wl = W.hh_single(4096, seed=1)
    _case(orc, wl["mechs"][0], wl["n_nodes"], wl["v0"], 3)


def test_noalloc_matches_oracle_and_cur_cnexp_two_calls(orc):
    wl = W.cortical_mix(20011, seed=31)
    for spec in (wl["mechs"][0], wl["mechs"][9], wl["mechs"][5]):
        _case(orc, spec, wl["n_nodes"], wl["v0"], 1)


def test_noalloc_matches_oracle_and_cur_kin9_two_calls(orc):
    wl = W.kin9_clamped(5003, seed=4)
    _case(orc, wl["mechs"][0], wl["n_nodes"], wl["v0"], 2)


def test_noalloc_reports_nonfinite_then_recovers():
    """A NaN voltage at one node makes that node's rhs non-finite: the call
    reports NMODL_ERR_NONFINITE; the next call on finite inputs returns OK
    (the latch starts at zero on every call)."""
    from paper_1905_02241_b300 import _lib
    wl = W.hh_single(300, seed=1)
    spec = wl["mechs"][0]
    p = np.ascontiguousarray(spec["params"], dtype=np.float64)
    n = spec["node_index"].size
    ni = to_dev(spec["node_index"])
    st = to_dev(np.full((3, n), 0.3))
    vb = wl["v0"].copy()
    vb[17] = np.nan
    st_ = torch.cuda.current_stream().cuda_stream
    for vin, want in ((vb, -5), (wl["v0"], 0)):
        v, r, d = to_dev(vin), to_dev(np.zeros(n)), to_dev(np.ones(n))
        torch.cuda.synchronize()
        if want:
            with pytest.raises(_lib.NmodlError) as e:
                _lib.nmodl_cur_noalloc(0, st_, W.TYPE_HH, n, ni.data_ptr(), n, p.ctypes.data,
                                       p.size, st.data_ptr(), n, v.data_ptr(), r.data_ptr(),
                                       d.data_ptr())
            assert e.value.status == want
        else:
            _lib.nmodl_cur_noalloc(0, st_, W.TYPE_HH, n, ni.data_ptr(), n, p.ctypes.data,
                                   p.size, st.data_ptr(), n, v.data_ptr(), r.data_ptr(),
                                   d.data_ptr())
            assert np.all(np.isfinite(r.cpu().numpy()))


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
