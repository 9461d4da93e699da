"""Timing of the FP64 CPU oracle on the host cores (test infrastructure:
used by bench.py's CPU baseline only).

The oracle runs unmodified; one process per core (a plain subprocess that
loads only the oracle) advances its own disjoint node shard of the same
network, and the throughput is the instance-steps of all shards over the
longest wall time.
"""
from __future__ import annotations

import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

_ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _n_instances(sub) -> int:
    return int(sum(m["node_index"].size for m in sub["mechs"]))


def time_shard(sub, dt: float, target_s: float, max_steps: int):
    """(instance-steps, seconds) of the oracle stepping `sub` for about
    target_s seconds (at most max_steps steps)."""
    from oracle import oracle as orc
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], sub["v0"])
          for m in sub["mechs"]]
    ninst = _n_instances(sub)
    t0 = time.perf_counter()
    orc.step(sub["mechs"], st, sub["v0"], sub["n_nodes"], dt, nsteps=2)
    per_step = (time.perf_counter() - t0) / 2
    k = max(1, min(max_steps, int(target_s / max(per_step, 1e-9))))
    t0 = time.perf_counter()
    orc.step(sub["mechs"], st, sub["v0"], sub["n_nodes"], dt, nsteps=k)
    return ninst * k, time.perf_counter() - t0


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _save(sub, path: str) -> None:
    arrs = {"v0": sub["v0"], "n_nodes": np.array(sub["n_nodes"])}
    for k, m in enumerate(sub["mechs"]):
        arrs[f"t{k}"] = np.array(m["type"])
        arrs[f"p{k}"] = np.asarray(m["params"])
        arrs[f"ni{k}"] = np.asarray(m["node_index"])
    np.savez(path, **arrs)


def _load(path: str):
    z = np.load(path)
    mechs = []
    k = 0
    while f"t{k}" in z:
        mechs.append(dict(type=int(z[f"t{k}"]), params=z[f"p{k}"], node_index=z[f"ni{k}"]))
        k += 1
    return dict(v0=z["v0"], n_nodes=int(z["n_nodes"]), mechs=mechs)


def _worker(path: str, dt: float, target_s: float, max_steps: int) -> None:
    steps, sec = time_shard(_load(path), dt, target_s, max_steps)
    print(json.dumps({"instance_steps": steps, "seconds": sec}), flush=True)


def time_parallel(subs, dt: float, target_s: float, max_steps: int, timeout_s: float = 300.0):
    """Aggregate instance-steps/s of one subprocess per shard."""
    with tempfile.TemporaryDirectory() as d:
        procs = []
        for k, sub in enumerate(subs):
            path = os.path.join(d, f"shard{k}.npz")
            _save(sub, path)
            code = (f"from oracle.timing import _worker; "
                    f"_worker({path!r}, {dt!r}, {target_s!r}, {max_steps!r})")
            env = dict(os.environ, PYTHONPATH=_ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
            procs.append(subprocess.Popen([sys.executable, "-c", code], cwd=_ROOT, env=env,
                                          stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                          text=True))
        res = []
        for p in procs:
            try:
                out, _ = p.communicate(timeout=timeout_s)
            except subprocess.TimeoutExpired:
                p.kill()
                raise
            res.append(json.loads(out.strip().splitlines()[-1]))
    total = sum(r["instance_steps"] for r in res)
    wall = max(r["seconds"] for r in res)
    return total / wall, wall
