"""Benchmark: mechanism instance-steps/s of the NMODL hot path on one B300.

Workload (default): the 10-type cortical channel mix on 2,000,000 isolated
compartments, plain FP64 (cnexp gates, analytic-conductance currents,
deterministic rhs/d accumulation, diagonal v update), dt = 0.025 ms.  One
bench "step" is one 200-time-step run of the whole network through
nmodl_step (5 fused launches of 40 steps, each replayed from a CUDA graph).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--precision fp64|mixed] [--nodes N]

Prints one JSON line.  Multi-GPU (torchrun): every rank simulates its own
network of the same size (weak scaling, no data-path collective; a barrier
and a max-reduction of the timings only).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1905_02241_b300 import workloads as W  # noqa: E402

DT, CM, NSTEPS = 0.025, 1.0, 200
METRIC = "mechanism instance-steps/s (state+cur)"

import bench_costs as C  # noqa: E402

# the algorithmic FP64 count of a step (FP64 pipe instructions of this
# design's minimal implementation; see bench_costs)
fp64_ops_per_step = C.fp64_ops_per_step


def bf16_peaks():
    """Measured dense bf16 tensor-core peaks (burst, sustained) in flop/s:
    the cuBLAS bf16 GEMM peaks measured on this GPU type and stored in
    MEASURED_PEAKS.json at the repository root when present, else the
    fallback figures of an earlier B300 measurement (1.8 and 1.4 PFLOP/s)."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        mp = json.load(open(path))
        return (mp["bf16_tflops"] * 1e12, mp["bf16_tflops_sustained"] * 1e12,
                "measured (MEASURED_PEAKS.json)")
    except (OSError, KeyError, ValueError):
        return 1.8e15, 1.4e15, "fallback (no measured peaks file)"


def issue_peak(dev: int) -> float:
    """Warp instructions per second the GPU can issue: one per cycle on each
    of an SM's four sub-partitions, at the maximum SM clock nvidia-smi
    reports (2,032 MHz on this GPU type if it cannot be read)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = 2032.0
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(dev), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True,
                             text=True, timeout=20).stdout.strip()
        mhz = float(out.splitlines()[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        pass
    return 4.0 * sms * mhz * 1e6


def n_instances(wl) -> int:
    return int(sum(m["node_index"].size for m in wl["mechs"]))


# ------------------------------------------------------------------ clocks

class ClockSampler:
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.proc = None
        self.path = None
        if not uuid:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", uuid, f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) >= 8:
                rows.append(f)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = max(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        loaded = [s for s in sm if s > 0.5 * mx] or sm
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, x in zip(names, r[4:8]) if x == "Active"})
        return {"sm_mhz": float(np.median(loaded)), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


# -------------------------------------------------------------- CPU oracle

def _subnet(wl, nodes):
    remap = -np.ones(wl["n_nodes"], dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    mechs = []
    for m in wl["mechs"]:
        keep = remap[m["node_index"]] >= 0
        mechs.append(dict(type=m["type"], params=m["params"],
                          node_index=remap[m["node_index"][keep]].astype(np.int32)))
    return dict(n_nodes=int(nodes.size), mechs=mechs, v0=wl["v0"][nodes])


# the one recipe of both the reference arm and the cpu_baseline leg: the
# FP64 oracle on the host's cores, one process per core (at most 128), each
# stepping its own shard of whole nodes of the same workload
ORACLE_SHARD_NODES = 20000
ORACLE_SHARD_SECONDS = 4.0


def oracle_on_cores(wl, nodes: int):
    """(instance-steps/s, processes, seconds, sample) of the oracle on the
    host's cores: all shards' instance-steps over the longest shard's wall
    time."""
    from oracle import timing as otiming
    shard = min(ORACLE_SHARD_NODES, nodes)
    cores = max(1, min(otiming.host_cores(), nodes // shard, 128))
    subs = [_subnet(wl, np.arange(k * shard, (k + 1) * shard)) for k in range(cores)]
    rate, el = otiming.time_parallel(subs, DT, ORACLE_SHARD_SECONDS, NSTEPS)
    sample = (f"{cores} processes (one per host core), each the oracle on its own "
              f"{shard}-node shard of the same network (whole nodes), up to {NSTEPS} steps "
              f"in about {ORACLE_SHARD_SECONDS:g} s")
    return rate, cores, el, sample


def time_oracle(wl, n_nodes_sample: int, target_s: float):
    from oracle import oracle as orc
    nodes = np.arange(min(n_nodes_sample, wl["n_nodes"]))
    sub = _subnet(wl, nodes)
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], sub["v0"])
          for m in sub["mechs"]]
    ninst = n_instances(sub)
    t0 = time.perf_counter()
    orc.step(sub["mechs"], st, sub["v0"], sub["n_nodes"], DT, nsteps=2)
    per_step = (time.perf_counter() - t0) / 2
    k = max(1, min(NSTEPS, int(target_s / max(per_step, 1e-9))))
    t0 = time.perf_counter()
    orc.step(sub["mechs"], st, sub["v0"], sub["n_nodes"], DT, nsteps=k)
    el = time.perf_counter() - t0
    desc = (f"first {sub['n_nodes']} nodes ({ninst} instances, whole nodes) of the "
            f"same network, {k} time steps, single thread")
    return ninst * k / el, desc, el


# --------------------------------------------------------------------- main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--nodes", type=int, default=2_000_000)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--tile-smem", type=int, default=0, help="fix the fused tile budget (bytes)")
    ap.add_argument("--block", type=int, default=0, help="fix the fused block size")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--forms", default="all",
                    help="comma list of hh,batched,kinetic,kin9_network,surrogate,"
                         "mixed_errors,pade,cable,ions; all; none")
    args = ap.parse_args()

    from paper_1905_02241_b300.sharding import aggregate, network_seed, rank_info
    rank, world, local = rank_info()
    config = {"workload": f"cortical 10-type cnexp mix, {args.nodes} nodes, "
                          f"{NSTEPS} steps of dt {DT} ms, {args.precision}",
              "nodes": args.nodes, "steps_per_bench_step": NSTEPS, "dt_ms": DT,
              "l2": "inputs larger than L2 (states and node_index > 126 MB)"}

    if args.impl == "reference":
        if rank != 0:
            return
        wl = W.cortical_mix(args.nodes, seed=2)
        rates = []
        for s in range(args.warmup + args.steps):
            r, cores, _, sample = oracle_on_cores(wl, args.nodes)
            if s >= args.warmup:
                rates.append(r)
        v = float(np.median(rates))
        sample += f" per step; median of {args.steps} steps"

        line = {"impl": "reference", "metric": METRIC, "value": v,
                "unit": "instance-steps/s", "n_gpus": args.gpus, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": None, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": dict(config, instances=n_instances(wl),
                               parallelism=f"replicas x{args.gpus}"),
                "cpu_baseline": {"value": v, "unit": "instance-steps/s", "cores": cores,
                                 "kind": "oracle", "sample": sample},
                "e2e": {"value": v, "unit": "instance-steps/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = local if world > 1 else 0
    torch.cuda.set_device(dev)
    from paper_1905_02241_b300 import _lib
    from paper_1905_02241_b300.api import NMODL_FP64, NMODL_MIXED, Context, Mechanism

    wl = W.cortical_mix(args.nodes, seed=network_seed(2, rank))
    prec = NMODL_FP64 if args.precision == "fp64" else NMODL_MIXED
    ctx = Context(dev, precision=prec, tile_smem=args.tile_smem, block=args.block)
    mechs = [Mechanism(ctx, m["type"], m["node_index"], wl["n_nodes"], m["params"])
             for m in wl["mechs"]]
    n = wl["n_nodes"]
    ninst = n_instances(wl)
    v = torch.tensor(wl["v0"], device=f"cuda:{dev}")
    rhs = torch.zeros(n, dtype=torch.float64, device=v.device)
    d = torch.zeros_like(rhs)
    for m in mechs:
        m.init(v)
    torch.cuda.synchronize()
    stream = ctx.stream

    def one():
        ctx.step(mechs, DT, CM, v, rhs, d, NSTEPS)

    for _ in range(args.warmup):
        one()
    assert ctx.sync() == 0
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
        uuid = uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:
        pass
    clocks = ClockSampler(uuid) if rank == 0 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        one()
    e1.record(stream)
    e1.synchronize()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop() if clocks else None
    assert ctx.sync() == 0
    value, ms = aggregate(ms, float(ninst) * NSTEPS * args.steps, dist, v.device)
    window = ctx.options.window
    launches_per_step = -(-NSTEPS // window)
    gpu_launches = launches_per_step * args.steps

    # roofline of the dominant kernel (the fused tile kernel: the whole step)
    launch_ms = ms / gpu_launches
    peak = _lib.nmodl_probe_peak(dev, 0)  # FP64 FMA lane-ops/s, measured here
    count = fp64_ops_per_step(wl) if prec == NMODL_FP64 else C.mixed_fp64_ops_per_step(wl)
    ops_launch = count * window
    roof = {"bound": "alu", "pipe": "fp64",
            "achieved": ops_launch / (launch_ms * 1e-3) / 1e12,
            "peak": peak / 1e12, "unit": "Tops/s (FP64 pipe instructions)",
            "peak_source": "measured DFMA probe (nmodl_probe_peak), this run",
            "ops_per_launch": ops_launch,
            "ops_per_instance_step": count / ninst,
            "what": ("FP64-pipe use: this design's minimal FP64 instruction count of the "
                     "step (exp, reciprocal and division at their 2-instruction cost here) "
                     "over the measured launch time, against the measured FP64 peak; "
                     "HBM is idle (traffic below) and the integer and FP32 pipes have "
                     "headroom, so the FP64 pipe is the bound" if prec == NMODL_FP64 else
                     "FP64 residue of the mixed step (node sums and updates) over the "
                     "launch time, against the measured FP64 peak")}
    roof["frac"] = roof["achieved"] / roof["peak"]
    if prec == NMODL_MIXED:
        # the mixed step keeps little FP64 work (the node update) and no pipe
        # near its peak: its bound is the SMs' instruction issue, at the
        # warp instructions per instance-step ncu counts on the 1M-node mix
        fp64_frac = roof["frac"]
        ins = C.MIXED_WARP_INSTR_PER_STEP * ninst * window
        roof = {"bound": "issue", "pipe": "issue",
                "achieved": ins / (launch_ms * 1e-3) / 1e12,
                "peak": issue_peak(dev) / 1e12, "unit": "T warp-instructions/s",
                "peak_source": "4 warp instructions per cycle per SM at the maximum SM clock",
                "ops_per_launch": ins,
                "ops_per_instance_step": C.MIXED_WARP_INSTR_PER_STEP,
                "what": ("issue use: the warp instructions the mixed step issues (ncu count on "
                         "the 1,000,000-node mix, per instance-step) over the launch time, "
                         "against one instruction per cycle per SM sub-partition"),
                "fp64_residue_frac": fp64_frac,
                "fp64_residue_ops_per_instance_step": count / ninst}
        roof["frac"] = roof["achieved"] / roof["peak"]
    if prec == NMODL_FP64:
        # the same speed against the FP64-pipe bound of routines written
        # entirely in FP64 (a yardstick that does not move with the design)
        full = C.fp64_ops_per_step(wl, C.ALL_FP64)
        roof["ops_per_instance_step_all_fp64"] = full / ninst
        roof["frac_vs_all_fp64_routines"] = (full * window / (launch_ms * 1e-3)) / peak
    # DRAM bytes per 40-step launch: dram__bytes_read.sum + dram__bytes_write.sum
    # of one ncu capture of the same kernel on the 1,000,000-node network
    # (11,548,985 instances), scaled to this network by its instance count
    per_1m = {NMODL_FP64: 310.7e6, NMODL_MIXED: 312.6e6}[prec]
    roof["traffic"] = per_1m * ninst / 11548985 if window == 40 else None
    roof["traffic_unit"] = "bytes per launch"
    roof["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                              "launch on the 1,000,000-node network, scaled by instances")
    roof["kernel"] = "k_fused_tiles<FP64>" if prec == NMODL_FP64 else "k_fused_tiles<MIXED>"

    # end to end through the C ABI with host buffers (pinned)
    e2e = None
    if not args.no_e2e:
        host_states = [torch.empty((m.n_states, m.n), dtype=torch.float64).pin_memory()
                       for m in mechs]
        for m, hs in zip(mechs, host_states):
            for k in range(m.n_states):
                _lib.nmodl_get_state(m.handle, k, hs[k].data_ptr())
        v_host = v.cpu().pin_memory()
        h2d = v_host.numel() * 8 + sum(hs.numel() * 8 for hs in host_states)
        ksteps = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(ksteps):
            v.copy_(v_host, non_blocking=True)
            for m, hs in zip(mechs, host_states):
                for k in range(m.n_states):
                    _lib.nmodl_set_state(m.handle, k, hs[k].data_ptr())
            ctx.step(mechs, DT, CM, v, rhs, d, NSTEPS)
            for m, hs in zip(mechs, host_states):
                for k in range(m.n_states):
                    _lib.nmodl_get_state(m.handle, k, hs[k].data_ptr())
            v_host.copy_(v, non_blocking=True)
            torch.cuda.synchronize()
        el = time.perf_counter() - t0
        e2e = {"value": world * ninst * NSTEPS * ksteps / el, "unit": "instance-steps/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(h2d),
               "steps": ksteps}

    cpu = None
    if rank == 0 and not args.no_cpu:
        r1, sample1, el1 = time_oracle(wl, 60000, 6.0)
        cpu = {"value": r1, "unit": "instance-steps/s", "cores": 1, "kind": "oracle",
               "sample": sample1, "seconds": round(el1, 2)}
        # the same oracle on the host's cores, by the reference arm's recipe
        rp, cores, elp, sample = oracle_on_cores(wl, args.nodes)
        if cores > 1:
            cpu.update({"value": rp, "cores": cores, "seconds": round(elp, 2),
                        "sample": f"{sample} (the reference arm's recipe); single thread: "
                                  f"{r1:.4g} on " + sample1,
                        "single_thread": r1})

    plan = ctx.plan(mechs)
    forms = None
    if rank == 0 and world == 1 and args.forms != "none":
        import bench_forms as F
        want = (["hh", "batched", "mixed_errors", "kinetic", "kin9_network", "surrogate", "pade",
                 "cable", "ions"]
                if args.forms == "all"
                else args.forms.split(","))
        forms = {}
        burst, sustained, src = bf16_peaks()
        peaks = {"fp64": peak, "fp32": _lib.nmodl_probe_peak(dev, 1),
                 "mufu_ex2": _lib.nmodl_probe_peak(dev, 2), "bf16_burst": burst,
                 "bf16_sustained": sustained, "bf16_source": src,
                 "issue": issue_peak(dev)}
        for name in want:
            t0 = time.perf_counter()
            forms[name] = getattr(F, name)(dev, peaks)
            forms[name]["seconds"] = round(time.perf_counter() - t0, 1)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "instance-steps/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if prec == NMODL_FP64 else "f32+f64",
                "data": "synthetic", "config": dict(config, instances=ninst,
                                                    parallelism=f"replicas x{world}"),
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": gpu_launches, "clocks": clk, "plan": plan,
                "forms": forms}
        print(json.dumps(line))
    for m in mechs:
        m.close()
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
