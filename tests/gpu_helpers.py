"""Shared helpers of the GPU parity tests: build the same seeded inputs for
the CUDA path (through the C ABI) and the CPU oracle, and compare."""
from __future__ import annotations

import numpy as np

TOL_FP64 = 1e-12  # relative, scale max(|x_ref|, 1e-3) for states


def torch_dev():
    import torch
    return torch.device("cuda:0")


def to_dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    if dtype is not None:
        t = t.to(dtype)
    return t.to(torch_dev())


def make_mechs(ctx, wl):
    from paper_1905_02241_b300.api import Mechanism
    return [Mechanism(ctx, m["type"], m["node_index"], wl["n_nodes"], m["params"])
            for m in wl["mechs"]]


def state_err(got, ref):
    """max |got - ref| / max(|ref|, 1e-3) over all entries."""
    got, ref = np.asarray(got), np.asarray(ref)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3)))


def node_scale(orc, wl, states, v, rhs0=None, d0=None):
    """Per-node sum of |terms| entering rhs and d (cancellation-safe scale)."""
    n = wl["n_nodes"]
    sr = np.zeros(n) if rhs0 is None else np.abs(rhs0).copy()
    sd = np.zeros(n) if d0 is None else np.abs(d0).copy()
    for m, s in zip(wl["mechs"], states):
        c, g = orc.mech_currents(m["type"], m["params"], m["node_index"], v, s)
        np.add.at(sr, m["node_index"], np.abs(c))
        np.add.at(sd, m["node_index"], np.abs(g))
    return sr, sd


def sub_network(wl, nodes):
    """The isolated sub-network on the given (sorted) node ids, renumbered."""
    nodes = np.asarray(nodes, dtype=np.int64)
    remap = -np.ones(wl["n_nodes"], dtype=np.int64)
    remap[nodes] = np.arange(nodes.size)
    mechs, sel = [], []
    for m in wl["mechs"]:
        keep = remap[m["node_index"]] >= 0
        sel.append(np.nonzero(keep)[0])
        mechs.append(dict(type=m["type"], params=m["params"],
                          node_index=remap[m["node_index"][keep]].astype(np.int32)))
    return dict(n_nodes=nodes.size, mechs=mechs), sel


def oracle_cable_cells(sub, nsteps):
    """Pool worker (CPU only): the oracle's INITIAL and nsteps cable steps of
    a sub-network of whole cells (dict of nodes, mechs, parent, ga, gb, v0)."""
    from oracle import oracle as orc
    st0 = [orc.mech_init(m["type"], m["params"], m["node_index"], sub["v0"])
           for m in sub["mechs"]]
    return orc.step_cable(sub["mechs"], st0, sub["v0"], sub["n_nodes"], sub["parent"],
                          sub["ga"], sub["gb"], 0.025, nsteps=nsteps)
