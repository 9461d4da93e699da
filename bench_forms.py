"""Measurements of the derived forms against the plain FP64 form on the
same GPU (used by bench.py), each with its roofline (bench_costs):

  hh       Hodgkin-Huxley on 4,096 isolated compartments, 1,000 steps, FP64

  batched  the 10-type mix over 64 independent networks of log-uniform size
           (10k..500k compartments), all types in one fused launch per
           40-step window replayed from a CUDA graph, autotuned tile/block
           shapes; MIXED precision vs FP64 on the same networks
  kinetic  the 9-state scheme on 1M clamped compartments: FP64 Newton vs
           FP32 LU + FP64 residual refinement
  surrogate the BF16 MLP stand-in (trained here on Newton-generated pairs) on
           4M clamped compartments vs the FP64 Newton solve, with fallback
           rate and final error against the Newton trajectory
  ions     ion current write-back (ina, ik, ica) with a 3-state scheme and a
           calcium buffer reading ica, on the ion-tagged cortical mix

Each entry reports instance-steps/s (state + cur), its ratio to the FP64
form and a roofline block: the algorithmic count per instance-step on the
unit that bounds it, achieved rate, measured peak and fraction.  Errors of
the mixed and surrogate forms are reported here against the FP64 GPU path;
the tests compare both with the FP64 CPU oracle.
"""
from __future__ import annotations

import time

import numpy as np
import torch

import bench_costs as C
from paper_1905_02241_b300 import _lib  # noqa: F401
from paper_1905_02241_b300 import workloads as W
from paper_1905_02241_b300.api import NMODL_FP64, NMODL_MIXED, Context, Mechanism

DT, CM = 0.025, 1.0


def _mechs(ctx, wl):
    return [Mechanism(ctx, m["type"], m["node_index"], wl["n_nodes"], m["params"])
            for m in wl["mechs"]]


def _time(fn, ctx, reps):
    ctx.check()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(reps):
        fn()
    e1.record(ctx.stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    ctx.check()
    return ms


def _ninst(wl):
    return int(sum(m["node_index"].size for m in wl["mechs"]))


def _roof(count, rate, peak, pipe, unit="Tops/s", what=""):
    """count: operations per instance-step on the bounding unit; rate:
    instance-steps/s; peak: the unit's measured operations/s."""
    ach = count * rate
    bound = "tensor" if pipe.startswith("bf16") else "issue" if pipe == "issue" else "alu"
    return {"bound": bound, "pipe": pipe,
            "ops_per_instance_step": count, "achieved": ach / 1e12, "peak": peak / 1e12,
            "unit": unit, "frac": ach / peak, "what": what}


def hh(dev, peaks, n=4096, nsteps=1000, reps=3):
    """Hodgkin-Huxley, one instance on each of n isolated compartments,
    v0 uniform in [-70, -60] mV, dt 0.025 ms, nsteps steps of nmodl_step
    (the single-HH gate-warp kernel, CUDA graphs per 40-step window), FP64.
    The problem fills only part of the GPU (one block of three warps, one
    per gate, on each of at most 148 SMs: three of the four sub-partitions
    of an SM, each with its own FP64 unit), so the roofline is given
    against the whole GPU and against the sub-partitions the blocks
    occupy."""
    wl = W.hh_single(n, seed=1)
    ctx = Context(dev)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ctx.step(mechs, DT, CM, v, rhs, d, nsteps)           # plan, autotune, graphs
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, reps)
    rate = n * nsteps * reps / (ms * 1e-3)
    plan = ctx.plan(mechs)
    count = C.fp64_ops_per_step(wl) / n
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    out = {"instances": n, "steps_per_run": nsteps, "fp64": rate, "plan": plan,
           "roofline": _roof(count, rate, peaks["fp64"], "fp64", what=(
               "FP64 pipe instructions per instance-step (bench_costs), whole-GPU peak"))}
    if plan["form"] == "hh_gate_warps":  # blocks of 3 warps on 3 of 4 sub-partitions
        busy = min(plan["tiles"], sms) * 3 / (4 * sms)
        out["roofline"]["occupied_sub_partitions"] = min(plan["tiles"], sms) * 3
        out["roofline"]["frac_of_occupied_sub_partitions"] = out["roofline"]["frac"] / busy
        out["ns_per_step"] = 1e9 * n / rate
        # the floor of a latency-bound step: one warp's FP64 instructions
        # per step, each holding its sub-partition's FP64 unit for one issue
        # interval (32 lanes / the unit's lane rate, from the measured peak)
        interval_ns = 1e9 * 32 * 4 * sms / peaks["fp64"]
        floor_ns = C.HH_WARP_FP64_PER_STEP * interval_ns
        out["latency_roofline"] = {
            "bound": "fp64_issue_chain", "fp64_warp_instructions_per_step": C.HH_WARP_FP64_PER_STEP,
            "fp64_issue_interval_ns": interval_ns, "floor_ns_per_step": floor_ns,
            "ns_per_step": out["ns_per_step"], "frac": floor_ns / out["ns_per_step"],
            "what": ("a step's floor: one gate warp's FP64 instructions per step (ncu) times "
                     "the FP64 issue interval of a sub-partition (from the measured FP64 peak); "
                     "the integer and FP32 parts of the chain come on top")}
    else:
        busy = min(plan["tiles"], sms) / sms
        out["roofline"]["frac_of_occupied_sms"] = out["roofline"]["frac"] / busy
        out["roofline"]["occupied_sms"] = min(plan["tiles"], sms)
    for m in mechs:
        m.close()
    ctx.close()
    return out


def batched(dev, peaks, steps=2, nsteps=200, scale=1.0):
    wl = W.batched_networks(64, seed=3, scale=scale)
    n, ninst = wl["n_nodes"], _ninst(wl)
    out = {"networks": 64, "nodes": n, "instances": ninst, "steps_per_run": nsteps}
    ctx = Context(dev, precision=NMODL_MIXED)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    t0 = time.perf_counter()
    ctx.step(mechs, DT, CM, v, rhs, d, nsteps)          # plan + autotune + graphs
    ctx.check()
    out["plan_seconds"] = round(time.perf_counter() - t0, 3)
    out["plan_mixed"] = ctx.plan(mechs)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, steps)
    out["mixed"] = ninst * nsteps * steps / (ms * 1e-3)
    ctx.set_options(precision=NMODL_FP64)
    ctx.step(mechs, DT, CM, v, rhs, d, 40)
    ctx.check()
    out["plan_fp64"] = ctx.plan(mechs)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, 40), ctx, 1)
    out["fp64"] = ninst * 40 / (ms * 1e-3)
    out["mixed_over_fp64"] = out["mixed"] / out["fp64"]
    out["launches_per_run"] = -(-nsteps // ctx.options.window)
    out["roofline_mixed"] = _roof(C.mixed_fp64_ops_per_step(wl) / ninst, out["mixed"],
                                  peaks["fp64"], "fp64", what=(
                                      "FP64 residue of the mixed step (v += dv per node; the node "
                                      "sums and the update run as float pairs on the FP32 "
                                      "pipe) per instance-step, against the measured FP64 peak"))
    out["roofline_fp64"] = _roof(C.fp64_ops_per_step(wl) / ninst, out["fp64"], peaks["fp64"],
                                 "fp64", what="FP64 pipe instructions per instance-step")
    if peaks.get("issue"):
        out["roofline_mixed_issue"] = _roof(
            C.MIXED_WARP_INSTR_PER_STEP, out["mixed"], peaks["issue"], "issue",
            unit="T warp-instructions/s", what=(
                "warp instructions issued per instance-step (measured by ncu on the 1M-node "
                "mix), against the SM issue peak: 4 per cycle per SM at the maximum SM clock; "
                "the mixed step has no pipe near its peak and is bound by issue and barriers"))
    for m in mechs:
        m.close()
    ctx.close()
    return out


def pade(dev, peaks, n_nodes=2_000_000, nsteps=200):
    """(1,1) Pade cnexp (Section 5.2 option) against exact cnexp, both FP64,
    on the cortical mix: throughput ratio and the state / voltage difference
    after nsteps from the same initial condition."""
    wl = W.cortical_mix(n_nodes, seed=2)
    ninst = _ninst(wl)
    out = {"nodes": n_nodes, "instances": ninst, "steps_per_run": nsteps}
    res = {}
    for name, flag in (("exact", 0), ("pade", 1)):
        ctx = Context(dev, cnexp_pade=flag)
        mechs = _mechs(ctx, wl)
        v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
        rhs = torch.zeros_like(v)
        d = torch.zeros_like(v)
        for m in mechs:
            m.init(v)
        ctx.step(mechs, DT, CM, v, rhs, d, nsteps)       # plan, graphs, result
        res[name] = (v.clone(), [m.states() for m in mechs if m.n_states])
        ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
        out[name] = ninst * nsteps / (ms * 1e-3)
        for m in mechs:
            m.close()
        ctx.close()
    (ve, se), (vp, sp) = res["exact"], res["pade"]
    out["pade_over_exact"] = out["pade"] / out["exact"]
    out["v_abs_mV_max"] = float((vp - ve).abs().max())
    out["v_abs_mV_median"] = float((vp - ve).abs().median())
    out["state_abs_max"] = float(max((a - b).abs().max() for a, b in zip(sp, se)))
    out["state_abs_mean"] = float(sum((a - b).abs().mean() for a, b in zip(sp, se)) / len(sp))
    return out


def cable(dev, peaks, n_cells=10000, nsteps=200):
    """The cortical mix on cells of 20..400 compartments with tree
    morphologies: FP64 steps with the per-cell tree solve against the same
    compartments isolated (fused step), instance-steps/s."""
    from paper_1905_02241_b300.api import Cable
    cab = W.cable_cells(n_cells, seed=7)
    wl = W.cortical_mix(cab["n_nodes"], seed=2)
    ninst = _ninst(wl)
    out = {"cells": n_cells, "nodes": cab["n_nodes"], "instances": ninst,
           "steps_per_run": nsteps}
    ctx = Context(dev)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    cb = Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    cb.step(mechs, DT, CM, v, rhs, d, 40)
    out["plan_cable"] = ctx.plan(mechs)
    ms = _time(lambda: cb.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["cable_fp64"] = ninst * nsteps / (ms * 1e-3)
    # the per-step launch sequence (the no_fuse option)
    ctx.set_options(no_fuse=1)
    cb.step(mechs, DT, CM, v, rhs, d, 40)
    ms = _time(lambda: cb.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["cable_per_step_launches_fp64"] = ninst * nsteps / (ms * 1e-3)
    ctx.set_options(no_fuse=0)
    ctx.step(mechs, DT, CM, v, rhs, d, 40)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["isolated_fused_fp64"] = ninst * nsteps / (ms * 1e-3)
    out["plan_isolated"] = ctx.plan(mechs)
    out["cable_over_isolated"] = out["cable_fp64"] / out["isolated_fused_fp64"]
    out["roofline"] = _roof(C.cable_fp64_ops_per_step(wl, cab["parent"]) / ninst,
                            out["cable_fp64"], peaks["fp64"], "fp64", what=(
                                "FP64 pipe instructions per instance-step with the tree "
                                "solve in place of the diagonal update"))
    cb.close()
    for m in mechs:
        m.close()
    ctx.close()
    return out


def kin9_network(dev, peaks, n_nodes=1_000_000, frac=0.25, nsteps=200):
    """The cortical mix on n_nodes compartments with the 9-state kinetic
    scheme on a seeded 25 % of them (one instance each, v not clamped): all
    mechanism types in the fused tile kernel (its KIN variant; in FP64 with
    the largest tiles, the shape the autotuner picks among the fused ones)
    against the per-mechanism launch sequence (no_fuse), FP64 and MIXED; and
    the FP64 form the autotuner picks when it may also choose the
    per-mechanism launches."""
    wl = W.cortical_mix(n_nodes, seed=2)
    ni = np.nonzero(W.Stream(2, 901).uniform(n_nodes) < frac)[0].astype(np.int32)
    wl["mechs"].append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(4, 401)),
                            node_index=ni, name="kin9"))
    ninst = _ninst(wl)
    out = {"nodes": n_nodes, "instances": ninst, "kin9_instances": int(ni.size),
           "steps_per_run": nsteps}
    for name, prec, opt in (("fused_fp64", NMODL_FP64, dict(tile_smem=1 << 30)),
                            ("per_mechanism_fp64", NMODL_FP64, dict(no_fuse=1)),
                            ("autotuned_fp64", NMODL_FP64, {}),
                            ("fused_mixed", NMODL_MIXED, {}),
                            ("per_mechanism_mixed", NMODL_MIXED, dict(no_fuse=1))):
        ctx = Context(dev, precision=prec, **opt)
        mechs = _mechs(ctx, wl)
        v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
        rhs = torch.zeros_like(v)
        d = torch.zeros_like(v)
        for m in mechs:
            m.init(v)
        ctx.step(mechs, DT, CM, v, rhs, d, 40)
        ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
        out[name] = ninst * nsteps / (ms * 1e-3)
        if name in ("fused_fp64", "autotuned_fp64", "fused_mixed"):
            out["plan_" + name] = ctx.plan(mechs)
        for m in mechs:
            m.close()
        ctx.close()
    out["fused_over_per_mechanism_fp64"] = out["fused_fp64"] / out["per_mechanism_fp64"]
    out["fused_over_per_mechanism_mixed"] = out["fused_mixed"] / out["per_mechanism_mixed"]
    iso = wl["mechs"][:-1]
    count = (C.fp64_ops_per_step(dict(n_nodes=n_nodes, mechs=iso))
             + C.kin9_fp64_ops(2.0) * ni.size) / ninst
    out["roofline_fused_fp64"] = _roof(count, out["fused_fp64"], peaks["fp64"], "fp64", what=(
        "FP64 pipe instructions per instance-step (cnexp types and the 9-state Newton solve "
        "with 2 updates)"))
    return out


def _ion_mechs(ctx, wl):
    return [Mechanism(ctx, m["type"], m["node_index"], wl["n_nodes"], m["params"],
                      ion=m.get("ion", 0)) for m in wl["mechs"]]


def ions(dev, peaks, n_nodes=2_000_000, nsteps=200):
    """USEION write-back and the small systems on the ion-tagged cortical mix
    (10 cnexp types writing ina/ik/ica, a 3-state potassium scheme on half
    of the nodes, one calcium buffer per node reading ica), all in the fused
    tile kernel:

      network_fp64 / network_mixed   whole steps with ion arrays registered
      network_per_mechanism_fp64     the same as per-mechanism launches
      no_buffer_ions_fp64            the same without the buffer
      no_buffer_no_ions_fp64         ... and without ion arrays: the cost of
                                     the ion write-back is the ratio
      cacum_state_*                  buffer Newton kernel alone (GB/s of its
                                     44 algorithmic bytes per instance)
      kin3_state_*                   3-state solve kernel alone
    All rates are instance-steps/s (the buffer counts as an instance)."""
    wl = W.cortical_ions(n_nodes, seed=8)
    nb = dict(wl, mechs=[m for m in wl["mechs"] if m["type"] != W.TYPE_CACUM])
    out = {"nodes": n_nodes, "instances": _ninst(wl), "instances_no_buffer": _ninst(nb),
           "steps_per_run": nsteps}
    dv = f"cuda:{dev}"
    v0 = torch.tensor(wl["v0"], device=dv)
    for name, net, prec, use_ions in (("network_fp64", wl, NMODL_FP64, True),
                                      ("network_mixed", wl, NMODL_MIXED, True),
                                      ("no_buffer_ions_fp64", nb, NMODL_FP64, True),
                                      ("no_buffer_no_ions_fp64", nb, NMODL_FP64, False)):
        ctx = Context(dev, precision=prec)
        arrs = [torch.zeros_like(v0) for _ in range(3)]
        if use_ions:
            ctx.set_ions(*arrs)
        mechs = _ion_mechs(ctx, net)
        v = v0.clone()
        rhs = torch.zeros_like(v)
        d = torch.zeros_like(v)
        for m in mechs:
            m.init(v)
        ctx.step(mechs, DT, CM, v, rhs, d, 40)
        ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
        out[name] = _ninst(net) * nsteps / (ms * 1e-3)
        if name == "network_fp64":
            cai = [m for m in mechs if m.type == W.TYPE_CACUM][0].states()[0]
            out["cai_mM_median"] = float(cai.median())
            out["cai_mM_max"] = float(cai.max())
            out["ica_nonzero_nodes"] = int((arrs[2] != 0).sum())
            out["plan_fused"] = bool(ctx.plan(mechs)["fused"])
        for m in mechs:
            m.close()
        ctx.close()
    # the per-mechanism launch sequence (the no_fuse option)
    ctx = Context(dev, no_fuse=1)
    arrs = [torch.zeros_like(v0) for _ in range(3)]
    ctx.set_ions(*arrs)
    mechs = _ion_mechs(ctx, wl)
    v = v0.clone()
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ctx.step(mechs, DT, CM, v, rhs, d, 40)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["network_per_mechanism_fp64"] = _ninst(wl) * nsteps / (ms * 1e-3)
    for m in mechs:
        m.close()
    ctx.close()
    out["fused_over_per_mechanism"] = out["network_fp64"] / out["network_per_mechanism_fp64"]
    out["ion_writeback_cost"] = out["no_buffer_no_ions_fp64"] / out["no_buffer_ions_fp64"]
    out["mixed_over_fp64"] = out["network_mixed"] / out["network_fp64"]
    out["roofline_fp64"] = _roof(C.fp64_ops_per_step(wl) / _ninst(wl), out["network_fp64"],
                                 peaks["fp64"], "fp64", what=(
                                     "FP64 pipe instructions per instance-step (cnexp types, "
                                     "3-state solve, buffer Newton with 4 updates)"))
    # kernels alone, 8M instances, one per node
    n = 8_000_000
    ni = torch.arange(n, dtype=torch.int32, device=dv)
    vk = torch.tensor(W.Stream(21, 1).uniform(n, -90.0, 40.0), device=dv)
    ica = -torch.tensor(W.Stream(21, 2).loguniform(n, 1e-4, 1.0), device=dv)
    reps = 20
    for prec, tag in ((NMODL_FP64, "fp64"), (NMODL_MIXED, "mixed")):
        ctx = Context(dev, precision=prec)
        ctx.set_ions(ica=ica)
        buf = Mechanism(ctx, W.TYPE_CACUM, ni, n, W.cacum_params())
        k3 = Mechanism(ctx, W.TYPE_KIN3, ni, n, W.kin3_params(W.Stream(8, 802)))
        for m in (buf, k3):
            m.init(vk)
            m.state(DT, vk)
            ms = _time(lambda: [m.state(DT, vk) for _ in range(reps)], ctx, 1)
            key = ("cacum_state_" if m is buf else "kin3_state_") + tag
            out[key] = n * reps / (ms * 1e-3)
            if m is buf:
                out[key + "_GBs"] = out[key] * 44 / 1e9
            else:
                out[key + "_GBs"] = out[key] * 60 / 1e9
            out[key + "_updates"] = m.stats()["newton_max"]
            m.close()
        ctx.close()
    return out


def mixed_errors(dev, peaks, n_nodes=2_000_000, nsteps=200):
    """Per-quantity difference of the MIXED fused step from the FP64 fused
    step on the whole cortical network after nsteps from the same initial
    state (the FP64 step itself agrees with the FP64 CPU oracle, which the
    tests check; they also compare the MIXED step with the oracle directly).
    States: max |difference| per type and gate; v in mV; rhs and d of the
    last step relative to the node's d (rhs against 200 mV x d); currents:
    per type, the per-node current of that type evaluated from each run's
    final states and v, max |difference| over nodes relative to the type's
    largest per-node current."""
    wl = W.cortical_mix(n_nodes, seed=2)
    dv = f"cuda:{dev}"
    res = {"steps": nsteps, "nodes": n_nodes, "instances": _ninst(wl)}
    runs = {}
    for name, prec in (("fp64", NMODL_FP64), ("mixed", NMODL_MIXED)):
        ctx = Context(dev, precision=prec)
        mechs = _mechs(ctx, wl)
        v = torch.tensor(wl["v0"], device=dv)
        rhs = torch.zeros_like(v)
        d = torch.zeros_like(v)
        for m in mechs:
            m.init(v)
        ctx.step(mechs, DT, CM, v, rhs, d, nsteps)
        ctx.check()
        runs[name] = (v, rhs, d, [m.states() for m in mechs], ctx, mechs)
    v64, r64, d64, s64, ctx64, mechs64 = runs["fp64"]
    vmx, rmx, dmx, smx, ctxmx, mechsmx = runs["mixed"]
    dv_abs = (vmx - v64).abs()
    res["v_abs_mV_max"] = float(dv_abs.max())
    res["v_abs_mV_median"] = float(dv_abs.median())
    res["d_rel_max"] = float(((dmx - d64).abs() / d64).max())
    res["rhs_rel_to_200mV_d_max"] = float(((rmx - r64).abs() / (200 * d64)).max())
    per_state, per_cur = {}, {}
    zero = torch.zeros_like(v64)
    for k, (spec, a64, amx) in enumerate(zip(W.CORTICAL_TYPES, s64, smx)):
        if a64.shape[0]:
            per_state[spec[0]] = [float(x) for x in (amx - a64).abs().max(dim=1).values]
        # the type's current per node from each run's states and v (FP64 call)
        m = mechs64[k]
        cur = []
        for st, vv in ((a64, v64), (amx, vmx)):
            if st.shape[0]:
                m.set_states(st)
            r = zero.clone()
            m.cur(vv, r, zero.clone())
            cur.append(r)
        ctx64.check()
        scale = float(cur[0].abs().max())
        per_cur[spec[0]] = float((cur[1] - cur[0]).abs().max()) / max(scale, 1e-300)
    res["state_abs_max"] = per_state
    res["current_rel_max"] = per_cur
    for name in runs:
        for m in runs[name][5]:
            m.close()
        runs[name][4].close()
    return res


def kinetic(dev, peaks, n=1_000_000, nsteps=200, steps=1):
    wl = W.kin9_clamped(n, seed=4)
    out = {"instances": n, "steps_per_run": nsteps}
    x0 = torch.tensor(wl["x0"], device=f"cuda:{dev}")
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for name, prec in (("fp64", NMODL_FP64), ("mixed", NMODL_MIXED)):
        ctx = Context(dev, precision=prec, clamp_v=1)
        (m,) = _mechs(ctx, wl)
        m.set_states(x0)
        ctx.step([m], DT, CM, v, rhs, d, 2)
        m.set_states(x0)
        ms = _time(lambda: ctx.step([m], DT, CM, v, rhs, d, nsteps), ctx, steps)
        out[name] = n * nsteps * steps / (ms * 1e-3)
        st = m.stats()
        out[name + "_updates_per_solve"] = st["newton_iters"] / max(1, st["calls"]) / n
        out[name + "_final"] = m.states()
        m.close()
        ctx.close()
    diff = (out.pop("mixed_final") - out.pop("fp64_final")).abs().sum(dim=0)
    out["mixed_over_fp64"] = out["mixed"] / out["fp64"]
    out["mixed_max_l1_vs_fp64"] = float(diff.max())
    out["roofline_fp64"] = _roof(C.kin9_fp64_ops(out["fp64_updates_per_solve"]), out["fp64"],
                                 peaks["fp64"], "fp64", what=(
                                     "FP64 pipe instructions per instance-step: rates, banded "
                                     "LU, Newton updates, current"))
    out["roofline_mixed"] = _roof(C.kin9_mixed_fp64_ops(out["mixed_updates_per_solve"]),
                                  out["mixed"], peaks["fp64"], "fp64", what=(
                                      "FP64 residue per instance-step: x - y and y += delta per "
                                      "update (the residual's rate terms and J's diagonal run as "
                                      "float pairs on the FP32 pipe), current"))
    return out


def surrogate(dev, peaks, n=4_000_000, nsteps=200, n_pairs=10_000_000, epochs=60):
    """The kinetic surrogate: FP64 Newton pairs, training (tensor-core
    kernels), then 200 gated steps on n clamped instances (instances above
    the 1e-4 residual fall back to the FP32-LU Newton with FP64 refinement)
    against the FP64 and FP32-LU Newton solves alone; the inference kernel
    alone (every prediction kept); rooflines of inference (tensor and
    special-function units) and of training (tensor)."""
    from paper_1905_02241_b300.surrogate import Surrogate, attach, make_training_pairs
    p = W.kin9_params(W.Stream(4, 401))
    out = {"instances": n, "steps_per_run": nsteps, "training_pairs": n_pairs,
           "epochs": epochs, "tolerance": 1e-4}
    ctx = Context(dev, clamp_v=1)
    t0 = time.perf_counter()
    batch = 8192
    sur = Surrogate(ctx, max_batch=batch)
    Ws, bs = W.mlp_init(7)
    sur.set_weights(Surrogate.pack(Ws, bs))
    X, T = make_training_pairs(ctx, sur, p, n_pairs, seed=6)
    torch.cuda.synchronize()
    out["pairs_seconds"] = round(time.perf_counter() - t0, 2)
    # torch loads its reduction kernels on first use (about a second), and
    # fit averages the loss record with one: not part of the training
    torch.zeros(2, device=X.device).mean().item()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    losses = sur.fit(X, T, epochs=epochs, batch=batch, lr=2e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    out["train_seconds"] = round(train_s, 2)
    out["final_loss"] = float(losses[-1])
    rows = (n_pairs // batch) * batch * epochs
    out["train_epoch_seconds"] = train_s / epochs
    out["train_optimiser_step_us"] = train_s / (rows / batch) * 1e6
    out["roofline_training"] = _roof(
        C.TRAIN_FLOPS_PER_ROW, rows / train_s, peaks["bf16_sustained"], "bf16_sustained",
        unit="TFLOP/s", what=("BF16 MMA flops per training row (forward, backward and "
                              "weight-gradient products, padded shapes) over the wall time of "
                              "the run (graph-replayed optimiser steps of 8,192 rows), "
                              "against the sustained bf16 peak (" + peaks["bf16_source"] + ")"))
    del X, T
    wl = W.kin9_clamped(n, seed=5)
    x0 = torch.tensor(wl["x0"], device=f"cuda:{dev}")
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    (m,) = _mechs(ctx, wl)
    ctx.step([m], DT, CM, v, rhs, d, 2)        # plan (autotuned) outside the timing
    m.set_states(x0)
    ms = _time(lambda: ctx.step([m], DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["newton_fp64"] = n * nsteps / (ms * 1e-3)
    ref = m.states()
    m.close()
    (m,) = _mechs(ctx, wl)
    attach(m, sur, 1e-4)
    ctx.step([m], DT, CM, v, rhs, d, 2)
    m.set_states(x0)
    fb_warm = m.stats()["fallback"]
    ms = _time(lambda: ctx.step([m], DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["surrogate"] = n * nsteps / (ms * 1e-3)
    st = m.stats()
    out["fallback_rate"] = (st["fallback"] - fb_warm) / (n * nsteps)
    err = (m.states() - ref).abs().sum(dim=0)
    out["final_max_l1_vs_newton"] = float(err.max())
    out["final_mean_l1_vs_newton"] = float(err.mean())
    out["surrogate_over_newton_fp64"] = out["surrogate"] / out["newton_fp64"]
    # (the fallback at this tolerance is the FP32-LU Newton with FP64
    # refinement; the comparison below is with that Newton alone)
    ctx.set_options(precision=NMODL_MIXED)
    # the inference kernel alone: every prediction kept (no fallback work)
    attach(m, sur, 1e30)
    m.set_states(x0)
    m.state(DT, v)
    reps = 10
    ms = _time(lambda: [m.state(DT, v) for _ in range(reps)], ctx, 1)
    out["surrogate_kernel_alone"] = n * reps / (ms * 1e-3)
    attach(m, None)
    ctx.step([m], DT, CM, v, rhs, d, 2)        # plan (autotuned) outside the timing
    m.set_states(x0)
    ms = _time(lambda: ctx.step([m], DT, CM, v, rhs, d, nsteps), ctx, 1)
    out["newton_mixed"] = n * nsteps / (ms * 1e-3)
    out["surrogate_over_newton_mixed"] = out["surrogate"] / out["newton_mixed"]
    for key, rate in (("kernel_alone", out["surrogate_kernel_alone"]),
                      ("end_to_end", out["surrogate"])):
        out["roofline_" + key] = _roof(
            C.MLP_FLOPS, rate, peaks["bf16_sustained"], "bf16_sustained", unit="TFLOP/s",
            what=("BF16 MMA flops of the MLP per instance-step (K and N padded to 16), "
                  "against the sustained bf16 peak (" + peaks["bf16_source"] + ")"))
        out["roofline_" + key]["frac_of_burst"] = C.MLP_FLOPS * rate / peaks["bf16_burst"]
        out["roofline_" + key]["mufu_frac"] = C.SUR_MUFU * rate / peaks["mufu_ex2"]
    m.close()
    sur.close()
    ctx.close()
    return out


def surrogate_kernel_case(dev=0, n=4_000_000, steps=3, tol=1e-4):
    """Profiling case of the fused surrogate kernel: n clamped instances,
    `steps` surrogate state updates with seeded (untrained) weights and the
    residual gate tol (inf keeps every prediction, timing the surrogate
    kernel alone); prints instance-steps/s."""
    from paper_1905_02241_b300.surrogate import Surrogate, attach
    wl = W.kin9_clamped(n, seed=5)
    ctx = Context(dev)
    sur = Surrogate(ctx, max_batch=256)
    Ws, bs = W.mlp_init(7)
    sur.set_weights(Surrogate.pack(Ws, bs))
    (m,) = _mechs(ctx, wl)
    m.set_states(torch.tensor(wl["x0"], device=f"cuda:{dev}"))
    attach(m, sur, tol)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    m.state(DT, v)
    ms = _time(lambda: [m.state(DT, v) for _ in range(steps)], ctx, 1)
    print({"instances": n, "steps": steps, "instance_steps_per_s": n * steps / (ms * 1e-3),
           "fallback": m.stats()["fallback"]})
    attach(m, None)
    m.close()
    sur.close()
    ctx.close()


def hh_case(dev=0, n=4096, nsteps=200):
    """Profiling case of the single-HH gate-warp kernel: the HH workload
    (n isolated compartments, one instance each, FP64), nsteps steps in
    windows of 40 (one launch each).  Prints instance-steps/s."""
    wl = W.hh_single(n, seed=1)
    ctx = Context(dev)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ctx.step(mechs, DT, CM, v, rhs, d, nsteps)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, nsteps), ctx, 1)
    print({"form": ctx.plan(mechs)["form"], "instance_steps_per_s": n * nsteps / (ms * 1e-3)})
    for m in mechs:
        m.close()
    ctx.close()


def ions_case(dev=0, n_nodes=1_000_000, windows=3):
    """Profiling case of the fused tile kernel's extended variant: the
    ion-tagged cortical mix (10 cnexp types writing ina/ik/ica, the 3-state
    scheme on half of the nodes, a calcium buffer per node) with ion arrays,
    FP64, autotuned on the first window, then `windows` timed windows of 40
    steps (one launch each).  Prints the plan and instance-steps/s."""
    wl = W.cortical_ions(n_nodes, seed=8)
    ctx = Context(dev)
    dv = f"cuda:{dev}"
    v = torch.tensor(wl["v0"], device=dv)
    arrs = [torch.zeros_like(v) for _ in range(3)]
    ctx.set_ions(*arrs)
    mechs = _ion_mechs(ctx, wl)
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ctx.step(mechs, DT, CM, v, rhs, d, 40)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, 40 * windows), ctx, 1)
    print({"plan": ctx.plan(mechs), "instance_steps_per_s": _ninst(wl) * 40 * windows / (ms * 1e-3)})
    for m in mechs:
        m.close()
    ctx.close()


def kin9_network_case(dev=0, n_nodes=1_000_000, windows=3, mixed=False, **opt):
    """Profiling case of the fused tile kernel's 9-state variant: the
    cortical mix on n_nodes with the 9-state scheme on a seeded 25 % of the
    nodes (the kin9_network form's workload), a first window (autotuned
    unless `opt` fixes the shape, e.g. autotune=0, tile_smem=216528,
    block=768), then `windows` timed windows of 40 steps.  Prints the plan
    and instance-steps/s."""
    wl = W.cortical_mix(n_nodes, seed=2)
    ni = np.nonzero(W.Stream(2, 901).uniform(n_nodes) < 0.25)[0].astype(np.int32)
    wl["mechs"].append(dict(type=W.TYPE_KIN9, params=W.kin9_params(W.Stream(4, 401)),
                            node_index=ni, name="kin9"))
    ctx = Context(dev, precision=NMODL_MIXED if mixed else NMODL_FP64, **opt)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs, d = torch.zeros_like(v), torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ctx.step(mechs, DT, CM, v, rhs, d, 40)
    ms = _time(lambda: ctx.step(mechs, DT, CM, v, rhs, d, 40 * windows), ctx, 1)
    print({"plan": ctx.plan(mechs), "instance_steps_per_s": _ninst(wl) * 40 * windows / (ms * 1e-3)})
    for m in mechs:
        m.close()
    ctx.close()


def training_case(dev=0, n_pairs=1 << 20, epochs=2, batch=8192):
    """Profiling case of the fused tensor-core training kernel: n_pairs
    FP64 Newton pairs of the 9-state scheme, `epochs` passes in minibatches
    of `batch` rows (one k_train_tiles + one k_grad_adam launch per
    optimiser step, replayed from a CUDA graph).  Prints optimiser steps/s
    and the BF16 MMA rate."""
    from paper_1905_02241_b300.surrogate import Surrogate, make_training_pairs
    p = W.kin9_params(W.Stream(4, 401))
    ctx = Context(dev)
    sur = Surrogate(ctx, max_batch=batch)
    Ws, bs = W.mlp_init(7)
    sur.set_weights(Surrogate.pack(Ws, bs))
    X, T = make_training_pairs(ctx, sur, p, n_pairs, seed=6)
    # torch loads its reduction kernels on first use (about a second), and
    # fit averages the loss record with one: not part of the training
    torch.zeros(2, device=X.device).mean().item()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    sur.fit(X, T, epochs=epochs, batch=batch, lr=2e-3)
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    steps = epochs * (n_pairs // batch)
    print({"optimiser_steps_per_s": steps / el,
           "bf16_tflops": steps * batch * C.TRAIN_FLOPS_PER_ROW / el / 1e12})
    sur.close()
    ctx.close()


def kernel_cases(dev=0):
    """Profiling case of the small-system, ion and cable kernels (seeded,
    synthetic): two calcium-buffer and two 3-state updates on 4M instances,
    one current update with ion write-back of each mechanism of the
    ion-tagged cortical mix on 500k nodes, and one 40-step window of the
    fused cable step on the benchmark's 10,000 cells (fixed 104 KB tiles of 512
    threads, two blocks per SM as the autotuner picks on the bench, no
    autotuning).  Prints instance-steps/s of each part."""
    from paper_1905_02241_b300.api import Cable
    dv = f"cuda:{dev}"
    out = {}
    n = 4_000_000
    ni = torch.arange(n, dtype=torch.int32, device=dv)
    vk = torch.tensor(W.Stream(21, 1).uniform(n, -90.0, 40.0), device=dv)
    ica = -torch.tensor(W.Stream(21, 2).loguniform(n, 1e-4, 1.0), device=dv)
    ctx = Context(dev)
    ctx.set_ions(ica=ica)
    buf = Mechanism(ctx, W.TYPE_CACUM, ni, n, W.cacum_params())
    k3 = Mechanism(ctx, W.TYPE_KIN3, ni, n, W.kin3_params(W.Stream(8, 802)))
    for m, key in ((buf, "cacum"), (k3, "kin3")):
        m.init(vk)
        ms = _time(lambda: [m.state(DT, vk) for _ in range(2)], ctx, 1)
        out[key + "_state"] = 2 * n / (ms * 1e-3)
        m.close()
    ctx.close()
    wl = W.cortical_ions(500_000, seed=8)
    nn = wl["n_nodes"]
    ctx = Context(dev)
    arrs = [torch.zeros(nn, dtype=torch.float64, device=dv) for _ in range(3)]
    ctx.set_ions(*arrs)
    mechs = [m for m in _ion_mechs(ctx, wl) if m.type != W.TYPE_CACUM]
    v = torch.tensor(wl["v0"], device=dv)
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    ms = _time(lambda: [m.cur(v, rhs, d) for m in mechs], ctx, 1)
    out["cur_ions"] = sum(m.n for m in mechs) / (ms * 1e-3)
    ctx.close()
    cab = W.cable_cells(10000, seed=7)
    wl = W.cortical_mix(cab["n_nodes"], seed=2)
    ctx = Context(dev, autotune=0, tile_smem=104 * 1024, block=512)
    mechs = _mechs(ctx, wl)
    v = torch.tensor(wl["v0"], device=dv)
    rhs = torch.zeros_like(v)
    d = torch.zeros_like(v)
    for m in mechs:
        m.init(v)
    cb = Cable(ctx, cab["parent"], cab["ga"], cab["gb"])
    ms = _time(lambda: cb.step(mechs, DT, CM, v, rhs, d, 40), ctx, 1)
    out["cable_fused"] = _ninst(wl) * 40 / (ms * 1e-3)
    out["cable_plan"] = ctx.plan(mechs)
    cb.close()
    ctx.close()
    print(out)


if __name__ == "__main__":
    import sys
    surrogate_kernel_case(n=int(sys.argv[1]) if len(sys.argv) > 1 else 4_000_000,
                          tol=float(sys.argv[2]) if len(sys.argv) > 2 else 1e-4)
