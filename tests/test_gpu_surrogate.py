"""GPU tests of the kinetic surrogate: the BF16 tensor-core MLP forward and
gradients against the FP64 CPU oracle (and against an emulation of the BF16
rounding points), training, the residual-gated fallback to Newton and the
gain of a trained network over the plain Newton solve."""
import numpy as np
import pytest

from paper_1905_02241_b300 import workloads as W
from gpu_helpers import make_mechs, state_err, to_dev

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def S():
    from paper_1905_02241_b300 import surrogate
    return surrogate


@pytest.fixture(scope="module")
def ctx():
    from paper_1905_02241_b300.api import Context
    c = Context(0)
    yield c


def _bf16(a):
    """Round float32 values to bfloat16 (nearest even), returned as float64."""
    a = np.asarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def _silu32(z):
    z = z.astype(np.float32)
    return (z / (np.float32(1) + np.exp(-z))).astype(np.float64)


def _emulate(Ws, bs, X):
    """Forward pass with the GPU's rounding points: bf16 inputs, weights and
    hidden activations; FP32 accumulation emulated in FP64."""
    h = _bf16(X.T)                      # (11, B)
    for li, (Wl, bl) in enumerate(zip(Ws, bs)):
        z = _bf16(Wl.astype(np.float32)) @ h + bl.astype(np.float32)[:, None]
        z = z.astype(np.float32).astype(np.float64)
        h = _bf16(_silu32(z)) if li < 3 else z
    return h


def _inputs(orc, n, seed):
    v, dt, x, _ = W.surrogate_samples(n, seed)
    return orc.surrogate_inputs(v, dt, x).T.astype(np.float32)   # (n, 11)


def test_forward_matches_oracle_and_bf16_emulation(S, ctx, orc):
    Ws, bs = W.mlp_init(3, out_scale=1.0)
    rng = np.random.default_rng(1)
    bs = [rng.normal(scale=0.1, size=b.shape) for b in bs]
    sur = S.Surrogate(ctx, max_batch=4096, weights=S.Surrogate.pack(Ws, bs))
    X = _inputs(orc, 1000, 3)
    Y = sur.forward(to_dev(X)).cpu().numpy().T            # (9, n)
    ref, _ = orc.mlp_forward(Ws, bs, X.T.astype(np.float64))
    emu = _emulate(Ws, bs, X)
    scale = np.max(np.abs(ref))
    # exp implementations differ (device __expf vs numpy), which flips some
    # bf16 roundings of hidden activations by one unit
    assert np.max(np.abs(Y - emu)) <= 5e-3 * scale, np.max(np.abs(Y - emu)) / scale
    rel = np.linalg.norm(Y - ref) / np.linalg.norm(ref)
    print(f"forward: rel L2 vs FP64 oracle {rel:.2e}, vs bf16 emulation "
          f"{np.max(np.abs(Y - emu)) / scale:.2e}")
    assert rel <= 2e-2
    sur.close()


@pytest.mark.parametrize("n,max_batch", [(512, 1024), (400, 400)])  # whole / partial last tile
def test_gradients_vs_oracle(S, ctx, orc, n, max_batch):
    Ws, bs = W.mlp_init(5, out_scale=1.0)
    sur = S.Surrogate(ctx, max_batch=max_batch, weights=S.Surrogate.pack(Ws, bs))
    X = _inputs(orc, n, 4)
    T = np.sin(np.arange(9 * n)).reshape(n, 9).astype(np.float32) * 0.3
    loss, g = sur.loss_grad(to_dev(X), to_dev(T))
    l_ref, gW, gb = orc.mlp_loss_grad(Ws, bs, X.T.astype(np.float64),
                                      T.T.astype(np.float64))
    assert abs(loss - l_ref) <= 2e-2 * l_ref
    gWg, gbg = S.Surrogate.unpack(g)
    for li in range(4):
        for a, b in ((gWg[li], gW[li]), (gbg[li], gb[li])):
            cos = float(np.sum(a * b) / (np.linalg.norm(a) * np.linalg.norm(b)))
            rel = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            assert cos >= 0.999 and rel <= 2e-2, (li, cos, rel)
    sur.close()


def test_weights_roundtrip(S, ctx):
    Ws, bs = W.mlp_init(9)
    w = S.Surrogate.pack(Ws, bs)
    sur = S.Surrogate(ctx, max_batch=256)
    sur.set_weights(w)
    np.testing.assert_array_equal(sur.get_weights(), w)
    sur.close()


def test_training_reduces_loss(S, ctx):
    p = W.kin9_params(W.Stream(4, 401))
    sur = S.Surrogate(ctx, max_batch=4096)
    Ws, bs = W.mlp_init(11)
    sur.set_weights(S.Surrogate.pack(Ws, bs))
    X, T = S.make_training_pairs(ctx, sur, p, 65536, seed=12)
    losses = sur.fit(X, T, epochs=6, batch=4096, lr=2e-3)
    print("training losses per epoch", losses)
    assert losses[-1] < losses[0] / 3
    sur.close()


def test_fit_replays_the_optimiser_step(S, ctx):
    """The graph-replayed training run equals the loop of single optimiser
    steps (same kernels; the learning rate and bias corrections computed on
    the device instead of the host)."""
    from paper_1905_02241_b300 import _lib
    import math
    p = W.kin9_params(W.Stream(4, 401))
    Ws, bs = W.mlp_init(13)
    a = S.Surrogate(ctx, max_batch=512, weights=S.Surrogate.pack(Ws, bs))
    b = S.Surrogate(ctx, max_batch=512, weights=S.Surrogate.pack(Ws, bs))
    X, T = S.make_training_pairs(ctx, a, p, 4096, seed=14)
    epochs, batch, lr, lr_min = 3, 512, 2e-3, 1e-4
    la = a.fit(X, T, epochs=epochs, batch=batch, lr=lr, lr_min=lr_min)
    spe = X.shape[0] // batch
    total = epochs * spe
    loss = torch.zeros(total, dtype=torch.float32, device="cuda:0")
    ctx.enter()
    for k in range(total):
        o = (k % spe) * batch
        rate = lr_min + 0.5 * (lr - lr_min) * (1 + math.cos(math.pi * k / total))
        _lib.nmodl_surrogate_train_step(b.handle, batch, X[o].data_ptr(), T[o].data_ptr(),
                                        rate, loss[k].data_ptr())
    ctx.leave()
    lb = loss.view(epochs, spe).mean(dim=1).cpu().numpy()
    np.testing.assert_allclose(la, lb, rtol=1e-4)
    wa, wb = a.get_weights(), b.get_weights()
    assert np.max(np.abs(wa - wb)) <= 1e-4 * np.max(np.abs(wb))
    assert ctx.sync() == 0
    a.close()
    b.close()


def _kin_setup(ctx, n, seed=4):
    wl = W.kin9_clamped(n, seed=seed)
    (m,) = make_mechs(ctx, wl)
    m.set_states(to_dev(wl["x0"]))
    return wl, m


@pytest.mark.parametrize("n", [1, 129, 151853])
def test_inference_kernel_vs_oracle(S, ctx, orc, n):
    """The tensor-core inference kernel with every prediction kept (gate
    above any residual) on one, a partial and many tiles per warpgroup with
    a ragged tail, against the FP64 oracle network + projection; the BF16
    network's increment error is bounded relative to the step scale s."""
    Ws, bs = W.mlp_init(9, out_scale=1.0)
    rng = np.random.default_rng(2)
    bs = [rng.normal(scale=0.1, size=b.shape) for b in bs]
    wl, m = _kin_setup(ctx, n, seed=8)
    spec = wl["mechs"][0]
    sur = S.Surrogate(ctx, max_batch=256, weights=S.Surrogate.pack(Ws, bs))
    S.attach(m, sur, 1e30)
    m.state(0.025, to_dev(wl["v0"]))
    got = m.states().cpu().numpy()
    assert m.stats()["fallback"] == 0
    idx = np.unique(np.concatenate([np.arange(0, n, 7), np.arange(max(0, n - 300), n)]))
    x = wl["x0"][:, idx]
    pred = orc.surrogate_step(Ws, bs, wl["v0"][idx], 0.025, x, spec["params"])
    s = np.array([np.abs(0.025 * orc.kin9_matrix(spec["params"], wl["v0"][c]) @ wl["x0"][:, c]).sum()
                  for c in idx])
    err = np.sum(np.abs(got[:, idx] - pred), axis=0)
    rel = err / np.maximum(s, 1e-30)
    print(f"n={n}: L1 error / s: max {rel.max():.2e}, median {np.median(rel):.2e}")
    assert np.all(err <= 3e-2 * s + 1e-6)
    assert np.median(rel) <= 5e-3
    assert np.max(np.abs(got.sum(axis=0) - 1.0)) <= 1e-5 and got.min() >= 0
    S.attach(m, None)
    sur.close()
    m.close()
    assert ctx.sync() == 0


def test_forced_fallback_equals_newton(S, ctx, orc):
    """A tolerance below FP32 rounding sends every instance to Newton."""
    wl, m = _kin_setup(ctx, 3001)
    sur = S.Surrogate(ctx, max_batch=256)                 # zero weights: x_hat = x
    S.attach(m, sur, 1e-30)
    m.state(0.025, to_dev(wl["v0"]))
    spec = wl["mechs"][0]
    ref = orc.mech_state(spec["type"], spec["params"], spec["node_index"], wl["v0"],
                         wl["x0"], 0.025)
    assert state_err(m.states().cpu().numpy(), ref) <= 1e-12
    st = m.stats()
    assert st["fallback"] == 3001 and st["surrogate_calls"] == 1
    assert ctx.sync() == 0
    S.attach(m, None)
    sur.close()


def _train(S, ctx, scaled, n_pairs, epochs, seed=13):
    p = W.kin9_params(W.Stream(4, 401))
    sur = S.Surrogate(ctx, max_batch=8192, scaled=scaled)
    Ws, bs = W.mlp_init(7)
    sur.set_weights(S.Surrogate.pack(Ws, bs))
    X, T = S.make_training_pairs(ctx, sur, p, n_pairs, seed=seed)
    losses = sur.fit(X, T, epochs=epochs, batch=8192, lr=2e-3)
    return sur, losses


@pytest.fixture(scope="module")
def trained(S, ctx):
    """The benchmark's training: 10M FP64 Newton pairs, 60 epochs."""
    sur, losses = _train(S, ctx, True, 10_000_000, 60)
    print("trained surrogate, last epoch losses", losses[-3:])
    yield sur
    sur.close()


def test_surrogate_error_bound_and_oracle(S, ctx, orc, trained):
    """Every instance ends within ||F||_1 <= 1e-4 of the exact implicit Euler
    step (P8); instances the surrogate kept match the oracle's surrogate."""
    wl, m = _kin_setup(ctx, 4096)
    spec = wl["mechs"][0]
    v = to_dev(wl["v0"])
    x = wl["x0"]
    # relax for a few Newton steps so that part of the population is slow
    for _ in range(20):
        m.state(0.025, v)
        x = orc.mech_state(spec["type"], spec["params"], spec["node_index"], wl["v0"],
                           x, 0.025)
    m.set_states(to_dev(x))
    S.attach(m, trained, 1e-4)
    m.state(0.025, v)
    got = m.states().cpu().numpy()
    exact = orc.mech_state(spec["type"], spec["params"], spec["node_index"], wl["v0"],
                           x, 0.025)
    err1 = np.sum(np.abs(got - exact), axis=0)
    fb = m.stats()["fallback"]
    print(f"one surrogate step: fallback {fb}/4096, max L1 error {err1.max():.2e}")
    assert err1.max() <= 1e-4 * (1 + 1e-3) + 1e-6
    kept = err1 > 1e-12
    assert kept.sum() > 0
    Ws, bs = S.Surrogate.unpack(trained.get_weights())
    idx = np.nonzero(kept)[0][:200]
    pred = orc.surrogate_step(Ws, bs, wl["v0"][idx], 0.025, x[:, idx], spec["params"])
    # BF16 network vs FP64 network: the difference is bounded by the scale
    # of the step; both sit within the residual bound of the exact step
    assert np.max(np.sum(np.abs(got[:, idx] - pred), axis=0)) <= 5e-4
    S.attach(m, None)
    assert ctx.sync() == 0


def test_surrogate_full_size_sampled_bound(S, ctx, orc, trained):
    """The surrogate benchmark's configuration: 4,000,000 clamped instances,
    one residual-gated surrogate step (kept predictions and Newton fallbacks
    together), checked on 2,000 sampled instances against the exact
    implicit Euler step: every one within the 1e-4 bound (P8), whatever the
    network's training."""
    n = 4_000_000
    wl, m = _kin_setup(ctx, n, seed=5)
    spec = wl["mechs"][0]
    S.attach(m, trained, 1e-4)
    m.state(0.025, to_dev(wl["v0"]))
    idx = np.unique(W.Stream(80, 1).integers(2000, 0, n - 1))
    got = m.states()[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy()
    exact = orc.mech_state(spec["type"], spec["params"], np.arange(idx.size, dtype=np.int32),
                           wl["v0"][idx], wl["x0"][:, idx], 0.025)
    err1 = np.sum(np.abs(got - exact), axis=0)
    st = m.stats()
    print(f"full size: fallback {st['fallback']}/{n}, sampled max L1 error {err1.max():.2e}")
    assert err1.max() <= 1e-4 * (1 + 1e-3) + 1e-6
    assert st["surrogate_calls"] == 1 and 0 <= st["fallback"] <= n
    S.attach(m, None)
    m.close()
    assert ctx.sync() == 0


def _timed_steps(m, v, steps):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        m.state(0.025, v)
    e1.record()
    e1.synchronize()
    return e0.elapsed_time(e1)


def test_surrogate_trajectory_vs_oracle_and_gain(S, ctx, orc, trained):
    """The surrogate benchmark's configuration: 4,000,000 clamped instances,
    200 residual-gated steps with the trained network.  What the network
    gains: under 10 % of the instance-steps fall back to Newton and the 200
    steps run faster than 200 FP64 Newton steps on the same instances.  Its
    error: on 1,000 sampled instances, against the FP64 oracle's Newton
    trajectory from the same initial states, the 1-norm error after 200
    steps stays within the sum of the per-step bounds (200 x 1e-4: the
    implicit Euler map is non-expansive in the 1-norm)."""
    n, steps = 4_000_000, 200
    wl, m = _kin_setup(ctx, n, seed=5)
    spec = wl["mechs"][0]
    v = to_dev(wl["v0"])
    S.attach(m, trained, 1e-4)
    m.state(0.025, v)                       # warm-up step, then the timed run
    m.set_states(to_dev(wl["x0"]))
    fb0 = m.stats()["fallback"]
    ms_sur = _timed_steps(m, v, steps)
    rate = (m.stats()["fallback"] - fb0) / (steps * n)
    idx = np.unique(W.Stream(82, 1).integers(1000, 0, n - 1))
    got = m.states()[:, torch.as_tensor(idx, device="cuda:0")].cpu().numpy()
    S.attach(m, None)
    m.set_states(to_dev(wl["x0"]))
    ms_newton = _timed_steps(m, v, steps)
    x = wl["x0"][:, idx]
    ni = np.arange(idx.size, dtype=np.int32)
    for _ in range(steps):
        x = orc.mech_state(spec["type"], spec["params"], ni, wl["v0"][idx], x, 0.025)
    err = np.sum(np.abs(got - x), axis=0)
    print(f"200 steps on 4M: fallback rate {rate:.4f}, surrogate {ms_sur:.1f} ms vs FP64 "
          f"Newton {ms_newton:.1f} ms ({ms_newton / ms_sur:.2f}x); L1 error vs FP64 oracle on "
          f"{idx.size} sampled instances: max {err.max():.2e}, mean {err.mean():.2e}")
    assert rate < 0.1
    assert ms_newton / ms_sur > 1.0
    assert err.max() <= steps * 1e-4
    m.close()
    assert ctx.sync() == 0


def _fallback_rate(S, ctx, sur, n=8000, steps=100):
    wl, m = _kin_setup(ctx, n, seed=6)
    S.attach(m, sur, 1e-4)
    v = to_dev(wl["v0"])
    for _ in range(steps):
        m.state(0.025, v)
    r = m.stats()["fallback"] / (steps * n)
    m.close()
    return r


def test_ablation_raw_state_inputs(S, ctx, trained):
    """The literal form (raw states in, increment out) against the scaled
    form: same data budget, fallback rate over a 100-step relaxation."""
    raw, losses = _train(S, ctx, False, 1 << 21, 8)
    r_raw = _fallback_rate(S, ctx, raw)
    r_scaled = _fallback_rate(S, ctx, trained)
    print(f"fallback rate: raw-state network {r_raw:.3f}, scaled network {r_scaled:.3f}")
    assert r_scaled < r_raw
    raw.close()


@pytest.mark.parametrize("clamp", [1, 0])
def test_network_step_form_matches_per_mechanism_launches(S, orc, clamp):
    """One 9-state mechanism with a surrogate and instance i on node i: the
    surrogate kernel runs the whole step (current at v_n, rhs, d, v_n+1,
    the gated state update and its fallback).  Against the per-mechanism
    launch sequence (no_fuse) of the same list and weights, over 12 steps in
    windows of 5, bit for bit: states, v, rhs, d and the fallback count; a
    list whose instance i is not on node i keeps the launches."""
    from paper_1905_02241_b300.api import Context, Mechanism
    n = 10007
    wl = W.kin9_clamped(n, seed=31)
    spec = wl["mechs"][0]
    Ws, bs = W.mlp_init(7)
    w = S.Surrogate.pack(Ws, bs)
    res = {}
    for form, nf in (("fused", 0), ("launches", 1)):
        ctx = Context(0, clamp_v=clamp, no_fuse=nf, window=5)
        sur = S.Surrogate(ctx, max_batch=256)
        sur.set_weights(w)
        m = Mechanism(ctx, spec["type"], spec["node_index"], n, spec["params"])
        m.set_states(to_dev(wl["x0"]))
        S.attach(m, sur, 1e-4)
        v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
        ctx.step([m], 0.025, 1.0, v, rhs, d, 12)
        assert ctx.sync() == 0
        res[form] = dict(plan=ctx.plan([m])["form"], v=v.cpu().numpy(), rhs=rhs.cpu().numpy(),
                         d=d.cpu().numpy(), x=m.states().cpu().numpy(), fb=m.stats()["fallback"])
        S.attach(m, None)
        m.close()
        sur.close()
        ctx.close()
    a, b = res["fused"], res["launches"]
    assert a["plan"] == "surrogate_step" and b["plan"] == "launches"
    assert a["fb"] == b["fb"] > 0
    for k in ("v", "rhs", "d", "x"):
        assert np.array_equal(a[k], b[k]), k
    if clamp:
        assert np.array_equal(a["v"], wl["v0"])
    else:
        assert not np.array_equal(a["v"], wl["v0"])
    # the one-step current against the oracle's (instance i on node i)
    ctx = Context(0, clamp_v=clamp)
    sur = S.Surrogate(ctx, max_batch=256)
    sur.set_weights(w)
    m = Mechanism(ctx, spec["type"], spec["node_index"], n, spec["params"])
    m.set_states(to_dev(wl["x0"]))
    S.attach(m, sur, 1e-4)
    v, rhs, d = to_dev(wl["v0"]), to_dev(np.zeros(n)), to_dev(np.zeros(n))
    ctx.step([m], 0.025, 1.0, v, rhs, d, 1)
    assert ctx.sync() == 0
    r_ref, d_ref = orc.mech_cur(spec["type"], spec["params"], spec["node_index"], wl["v0"],
                                wl["x0"], np.zeros(n), np.zeros(n))
    np.testing.assert_allclose(rhs.cpu().numpy(), r_ref, rtol=1e-12, atol=1e-300)
    np.testing.assert_allclose(d.cpu().numpy(), d_ref + 1e-3 / 0.025, rtol=1e-12)
    S.attach(m, None)
    m.close()
    # not instance i on node i: the launches
    ni = np.arange(n, dtype=np.int32)
    ni[5] = 4
    m = Mechanism(ctx, spec["type"], ni, n, spec["params"])
    m.set_states(to_dev(wl["x0"]))
    S.attach(m, sur, 1e-4)
    ctx.step([m], 0.025, 1.0, v, rhs, d, 1)
    assert ctx.sync() == 0 and ctx.plan([m])["form"] == "launches"
    S.attach(m, None)
    m.close()
    sur.close()
    ctx.close()
