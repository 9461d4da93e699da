"""Seeded synthetic inputs for the mechanism hot path.

This module only draws numbers: node indices, per-type parameter blocks,
initial voltages and initial kinetic states.  It holds none of the
mechanism arithmetic (no rates, no integration, no reductions), so both the
CUDA path and the CPU oracle can consume its arrays without sharing method
code.

Random numbers come from SplitMix64 (Steele, Lea and Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014) used as a
counter-based generator: value k of stream s is mix64(key(seed, s) +
(k + 1) * GAMMA).

Parameter block layouts (double precision, one block per mechanism type):

  HH (7):     gnabar, gkbar, gl [S/cm2], ena, ek, el [mV], celsius [degC]
  CNEXP (33): n_gates, gbar [S/cm2], e [mV], q10, celsius, t0,
              then 3 gate slots of 9 values:
              power, alpha_form, alpha_A, alpha_vh, alpha_k,
                     beta_form,  beta_A,  beta_vh,  beta_k
              forms: 0 = EXP      A*exp(u)
                     1 = SIGMOID  A/(1+exp(-u))
                     2 = LINOID   A*u/(1-exp(-u))
              with u = (v - vh)/k, A in 1/ms, vh and k in mV.
  KIN9 (51):  gbar [S/cm2], e [mV], open state index, then for each of the
              12 lattice edges (see KIN9_EDGES) a_f, b_f, a_b, b_b with the
              forward rate a_f*exp(b_f*v) and backward rate a_b*exp(-b_b*v).
  KIN3 (15):  gbar, e, open state index, then a_f, b_f, a_b, b_b for the
              edges (0,1), (1,2), (0,2).
  CACUM (6):  k [mM/ms per mA/cm2], tau [ms], cai0 [mM], kf [1/(mM ms)],
              kb [1/ms], btot [mM] of the calcium buffer.

Ion tags (USEION WRITE of the whole current): 0 none, 1 na, 2 k, 3 ca.
"""
from __future__ import annotations

import numpy as np

MASK64 = np.uint64(0xFFFFFFFFFFFFFFFF)
GAMMA = np.uint64(0x9E3779B97F4A7C15)

TYPE_HH = 1
TYPE_CNEXP = 2
TYPE_KIN9 = 3

TYPE_CACUM = 4
TYPE_KIN3 = 5
ION_NONE, ION_NA, ION_K, ION_CA = 0, 1, 2, 3

HH_NPARAM = 7
CNEXP_NPARAM = 33
CNEXP_GATE_BASE = 6
CNEXP_GATE_STRIDE = 9
KIN9_NPARAM = 51
KIN3_NPARAM = 15
CACUM_NPARAM = 6
FARADAY = 96485.33212  # C/mol

FORM_EXP, FORM_SIGMOID, FORM_LINOID = 0, 1, 2

# 3x3 lattice of kinetic states (a, b), index 3a+b; edges join lattice
# neighbours, listed as (lower index, higher index).  Horizontal edges first.
KIN9_EDGES = tuple(
    [(3 * a + b, 3 * a + b + 1) for a in range(3) for b in range(2)]
    + [(3 * a + b, 3 * (a + 1) + b) for a in range(2) for b in range(3)]
)
KIN9_OPEN = 6  # state (2, 0)


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= np.uint64(0xBF58476D1CE4E5B9)
        z ^= z >> np.uint64(27)
        z *= np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(31)
    return z


def _key(seed: int, stream: int) -> np.uint64:
    with np.errstate(over="ignore"):
        base = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) * GAMMA + np.uint64(
            (stream * 0xD1B54A32D192ED03) & 0xFFFFFFFFFFFFFFFF)
    return _mix64(np.array([base], dtype=np.uint64))[0]


class Stream:
    """One counter-based SplitMix64 stream; draws advance an internal counter."""

    def __init__(self, seed: int, stream: int):
        self.key = _key(seed, stream)
        self.counter = 0

    def u64(self, n: int) -> np.ndarray:
        k = np.arange(self.counter + 1, self.counter + 1 + n, dtype=np.uint64)
        self.counter += n
        with np.errstate(over="ignore"):
            return _mix64(self.key + k * GAMMA)

    def uniform(self, n: int, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
        u = (self.u64(n) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
        return lo + (hi - lo) * u

    def loguniform(self, n: int, lo: float, hi: float) -> np.ndarray:
        return np.exp(self.uniform(n, np.log(lo), np.log(hi)))

    def integers(self, n: int, lo: int, hi: int) -> np.ndarray:
        """Uniform integers in [lo, hi] (inclusive)."""
        span = hi - lo + 1
        return lo + (self.u64(n) % np.uint64(span)).astype(np.int64)

    def dirichlet(self, n: int, dim: int, alpha: float = 1.0) -> np.ndarray:
        """n points on the simplex, shape (dim, n), Dirichlet(alpha).

        alpha = 1 uses exponential variates; other alpha use numpy's gamma
        sampler seeded from this stream (input generation only).
        """
        if alpha == 1.0:
            u = self.uniform(n * dim)
            g = -np.log1p(-u).reshape(dim, n)
        else:
            rng = np.random.Generator(np.random.PCG64(int(self.u64(1)[0])))
            g = rng.gamma(alpha, 1.0, size=(dim, n))
            g = np.maximum(g, 1e-300)
        return g / g.sum(axis=0, keepdims=True)


# --------------------------------------------------------------------------
# parameter blocks
# --------------------------------------------------------------------------

def hh_params(gnabar=0.12, gkbar=0.036, gl=0.0003, ena=50.0, ek=-77.0,
              el=-54.3, celsius=6.3) -> np.ndarray:
    return np.array([gnabar, gkbar, gl, ena, ek, el, celsius], dtype=np.float64)


def cnexp_params(gbar: float, e: float, gates, q10: float = 3.0,
                 celsius: float = 6.3, t0: float = 6.3) -> np.ndarray:
    """gates: list of (power, (fa, Aa, vha, ka), (fb, Ab, vhb, kb))."""
    p = np.zeros(CNEXP_NPARAM, dtype=np.float64)
    if len(gates) > 3:
        raise ValueError("at most 3 gates")
    p[0] = len(gates)
    p[1], p[2], p[3], p[4], p[5] = gbar, e, q10, celsius, t0
    for g, (power, a, b) in enumerate(gates):
        o = CNEXP_GATE_BASE + CNEXP_GATE_STRIDE * g
        p[o] = power
        p[o + 1:o + 5] = a
        p[o + 5:o + 9] = b
    return p


def kin9_params(s: Stream, gbar: float = 0.12, e: float = 50.0) -> np.ndarray:
    p = np.zeros(KIN9_NPARAM, dtype=np.float64)
    p[0], p[1], p[2] = gbar, e, KIN9_OPEN
    af = s.loguniform(12, 0.05, 5.0)
    bf = s.uniform(12, 0.01, 0.04)
    ab = s.loguniform(12, 0.05, 5.0)
    bb = s.uniform(12, 0.01, 0.04)
    for k in range(12):
        p[3 + 4 * k:3 + 4 * k + 4] = (af[k], bf[k], ab[k], bb[k])
    return p


def kin3_params(s: Stream, gbar: float = 0.01, e: float = -85.0, open_state: int = 2,
                chain: bool = False) -> np.ndarray:
    """3-state scheme with seeded rates (the 9-state scheme's ranges);
    chain=True leaves the (0,2) edge out (a linear C-O-I chain)."""
    p = np.zeros(KIN3_NPARAM, dtype=np.float64)
    p[0], p[1], p[2] = gbar, e, open_state
    af = s.loguniform(3, 0.05, 5.0)
    bf = s.uniform(3, 0.01, 0.04)
    ab = s.loguniform(3, 0.05, 5.0)
    bb = s.uniform(3, 0.01, 0.04)
    for k in range(3):
        p[3 + 4 * k:3 + 4 * k + 4] = (af[k], bf[k], ab[k], bb[k])
    if chain:
        p[3 + 8:3 + 12] = (0.0, 0.0, 0.0, 0.0)
    return p


def cacum_params(depth_um: float = 0.1, tau: float = 200.0, cai0: float = 5e-5,
                 kf: float = 100.0, kb: float = 0.1, btot: float = 0.05) -> np.ndarray:
    """Calcium buffer in a submembrane shell of depth_um: an inward ica of
    1 mA/cm2 adds 1/(2 F depth) mM/ms (unit conversion only)."""
    k = 1.0 / (2.0 * FARADAY * depth_um * 1e-4)
    return np.array([k, tau, cai0, kf, kb, btot], dtype=np.float64)


# Ten channel templates of the cortical-style mix: name, reversal potential
# and the gates as (power, activating?) pairs.  Rate forms and constants are
# drawn per gate from the seed.
CORTICAL_TYPES = (
    ("NaT", 50.0, ((3, True), (1, False), (1, False))),
    ("NaP", 50.0, ((1, True),)),
    ("KT", -85.0, ((4, True), (1, False), (1, False))),
    ("KP", -85.0, ((2, True), (1, False))),
    ("Kv3", -85.0, ((1, True),)),
    ("Ih", -45.0, ((1, False),)),
    ("CaHVA", 120.0, ((2, True), (1, False))),
    ("CaLVA", 120.0, ((2, True), (1, False))),
    ("SK", -85.0, ((1, True),)),
    ("leak", -70.0, ()),
)


def _random_rate(s: Stream, increasing: bool, slow: bool):
    form = int(s.integers(1, 0, 2)[0])
    A = float(s.loguniform(1, 0.01, 1.0)[0])
    if slow:
        A *= 0.05
    vh = float(s.uniform(1, -70.0, -20.0)[0])
    k = float(s.uniform(1, 5.0, 30.0)[0])
    # u = (v - vh)/k grows with v for k > 0; every form increases with u.
    if not increasing:
        k = -k
    return (float(form), A, vh, k)


def cortical_type_params(seed: int):
    """Parameter blocks of the ten cnexp channel types (one per template)."""
    s = Stream(seed, 101)
    blocks = []
    for name, e, gates in CORTICAL_TYPES:
        gbar = float(s.loguniform(1, 1e-5, 1e-1)[0])
        q10 = float(s.uniform(1, 2.0, 3.0)[0])
        spec = []
        for power, act in gates:
            slow = name in ("SK", "Ih")
            a = _random_rate(s, act, slow)
            b = _random_rate(s, not act, slow)
            spec.append((power, a, b))
        # celsius == t0: the temperature factor is exactly 1
        blocks.append(cnexp_params(gbar, e, spec, q10=q10, celsius=6.3, t0=6.3))
    return blocks


def _type_node_index(s: Stream, node_ids: np.ndarray, frac: float,
                     kmax: int) -> np.ndarray:
    sel = node_ids[s.uniform(node_ids.size) < frac]
    k = s.integers(sel.size, 1, kmax)
    return np.repeat(sel, k).astype(np.int32)


def cortical_mix(n_nodes: int, seed: int = 2, kmax: int = 3,
                 v_lo: float = -90.0, v_hi: float = 40.0):
    """The 10-type cnexp channel mix on n_nodes isolated compartments.

    Type t sits on a random fraction p_t ~ U[0.2, 1] of the nodes with
    k ~ U{1..kmax} instances per selected node; node_index is sorted.
    Returns dict(v0, mechs=[dict(type, params, node_index, name)]).
    """
    blocks = cortical_type_params(seed)
    s = Stream(seed, 102)
    nodes = np.arange(n_nodes, dtype=np.int64)
    mechs = []
    for (name, _, _), p in zip(CORTICAL_TYPES, blocks):
        frac = float(s.uniform(1, 0.2, 1.0)[0])
        ni = _type_node_index(s, nodes, frac, kmax)
        mechs.append(dict(type=TYPE_CNEXP, params=p, node_index=ni, name=name))
    v0 = Stream(seed, 103).uniform(n_nodes, v_lo, v_hi)
    return dict(v0=v0, mechs=mechs, n_nodes=n_nodes)


# ion carried by each cortical template's current
CORTICAL_IONS = {"NaT": ION_NA, "NaP": ION_NA, "KT": ION_K, "KP": ION_K, "Kv3": ION_K,
                 "Ih": ION_NONE, "CaHVA": ION_CA, "CaLVA": ION_CA, "SK": ION_K,
                 "leak": ION_NONE}


def cortical_ions(n_nodes: int, seed: int = 8, kmax: int = 3, kin3_frac: float = 0.5):
    """The cortical mix with ion tags (sodium, potassium and calcium
    channels write ina, ik, ica), plus a 3-state potassium channel on a
    kin3_frac fraction of the nodes and one calcium buffer per node that
    reads ica.  Returns dict(v0, mechs, n_nodes); mechs carry "ion"."""
    net = cortical_mix(n_nodes, seed=seed, kmax=kmax)
    for m in net["mechs"]:
        m["ion"] = CORTICAL_IONS[m["name"]]
    s = Stream(seed, 801)
    nodes = np.arange(n_nodes, dtype=np.int64)
    ni3 = nodes[s.uniform(n_nodes) < kin3_frac].astype(np.int32)
    net["mechs"].append(dict(type=TYPE_KIN3, params=kin3_params(Stream(seed, 802)),
                             node_index=ni3, name="K3state", ion=ION_K))
    net["mechs"].append(dict(type=TYPE_CACUM, params=cacum_params(),
                             node_index=nodes.astype(np.int32), name="cacum",
                             ion=ION_NONE))
    return net


def hh_single(n_nodes: int = 4096, seed: int = 1):
    """HH on n_nodes isolated compartments, one instance each."""
    v0 = Stream(seed, 1).uniform(n_nodes, -70.0, -60.0)
    ni = np.arange(n_nodes, dtype=np.int32)
    return dict(v0=v0, n_nodes=n_nodes,
                mechs=[dict(type=TYPE_HH, params=hh_params(), node_index=ni,
                            name="hh")])


def network_sizes(n_networks: int = 64, seed: int = 3, lo: float = 1e4,
                  hi: float = 5e5, scale: float = 1.0) -> np.ndarray:
    s = Stream(seed, 301)
    sz = np.floor(s.loguniform(n_networks, lo, hi) * scale).astype(np.int64)
    return np.maximum(sz, 1)


def batched_networks(n_networks: int = 64, seed: int = 3, size_lo: float = 1e4,
                     size_hi: float = 5e5, scale: float = 1.0, kmax: int = 3,
                     type_seed: int = 2):
    """Independent networks of uneven size carrying the 10-type mix.

    The channel parameter blocks are shared (drawn from type_seed); each
    network draws its own type coverage.  Networks occupy consecutive node
    ranges [offsets[k], offsets[k+1]) of one concatenated node array.
    """
    sizes = network_sizes(n_networks, seed, size_lo, size_hi, scale)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    blocks = cortical_type_params(type_seed)
    s = Stream(seed, 302)
    per_type = [[] for _ in CORTICAL_TYPES]
    for k in range(n_networks):
        nodes = np.arange(offsets[k], offsets[k + 1], dtype=np.int64)
        for t in range(len(CORTICAL_TYPES)):
            frac = float(s.uniform(1, 0.2, 1.0)[0])
            per_type[t].append(_type_node_index(s, nodes, frac, kmax))
    mechs = []
    for t, (name, _, _) in enumerate(CORTICAL_TYPES):
        ni = np.concatenate(per_type[t]).astype(np.int32)
        mechs.append(dict(type=TYPE_CNEXP, params=blocks[t], node_index=ni,
                          name=name))
    n_nodes = int(offsets[-1])
    v0 = Stream(seed, 303).uniform(n_nodes, -90.0, 40.0)
    return dict(v0=v0, mechs=mechs, n_nodes=n_nodes, offsets=offsets)


def kin9_clamped(n: int, seed: int = 4, rate_seed: int = 4):
    """KIN9 lattice scheme, one instance per node, v clamped per node.

    Initial states are Dirichlet(1) points on the simplex (shape (9, n)).
    """
    p = kin9_params(Stream(rate_seed, 401))
    v = Stream(seed, 402).uniform(n, -100.0, 60.0)
    x0 = Stream(seed, 403).dirichlet(n, 9, 1.0)
    ni = np.arange(n, dtype=np.int32)
    return dict(v0=v, n_nodes=n, x0=x0,
                mechs=[dict(type=TYPE_KIN9, params=p, node_index=ni,
                            name="kin9")])


def surrogate_samples(n: int, seed: int = 6, v_lo=-100.0, v_hi=60.0,
                      dt_lo=0.0125, dt_hi=0.05):
    """(v, dt, x, lam) training inputs: x is an equal mixture of Dirichlet(1)
    and Dirichlet(0.2) points, shape (9, n); lam (n,) is 0 for two thirds
    of the samples and 1 - 10^U[-5, 0] for the rest (the weight with which
    the consumer pulls those samples towards the stationary distribution at
    their v, i.e. states near the end of a relaxation)."""
    s = Stream(seed, 601)
    v = s.uniform(n, v_lo, v_hi)
    dt = s.uniform(n, dt_lo, dt_hi)
    n1 = n // 2
    x = np.concatenate([Stream(seed, 602).dirichlet(n1, 9, 1.0),
                        Stream(seed, 603).dirichlet(n - n1, 9, 0.2)], axis=1)
    perm = np.argsort(Stream(seed, 604).u64(n), kind="stable")
    lam = np.where(Stream(seed, 605).uniform(n) < 1.0 / 3.0,
                   1.0 - 10.0 ** Stream(seed, 606).uniform(n, -5.0, 0.0), 0.0)
    return v, dt, np.ascontiguousarray(x[:, perm]), lam


def mlp_init(seed: int, widths=(11, 128, 128, 128, 9), out_scale: float = 0.1):
    """He-uniform initial weights (row-major [out][in]) and zero biases."""
    s = Stream(seed, 701)
    Ws, bs = [], []
    for li in range(len(widths) - 1):
        fi, fo = widths[li], widths[li + 1]
        lim = np.sqrt(6.0 / fi)
        if li == len(widths) - 2:
            lim *= out_scale
        Ws.append(s.uniform(fo * fi, -lim, lim).reshape(fo, fi))
        bs.append(np.zeros(fo))
    return Ws, bs


def cable_cells(n_cells: int, seed: int = 7, size_lo: int = 20, size_hi: int = 400,
                branch_p: float = 0.15):
    """Tree morphologies of n_cells cells on consecutive node ranges.

    parent[i] = -1 at the root of each cell; otherwise the previous node
    (unbranched run) or, with probability branch_p, a random earlier node of
    the same cell (a branch point).  ga ~ logU[0.5, 50] S/cm2 per unit area
    of the node, gb = ga * r with the area ratio r ~ U[0.5, 2].
    Returns dict(parent, ga, gb, offsets)."""
    s = Stream(seed, 801)
    sizes = s.integers(n_cells, size_lo, size_hi)
    offsets = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    n = int(offsets[-1])
    parent = np.empty(n, dtype=np.int32)
    u = s.uniform(n)
    r = s.uniform(n)
    for c in range(n_cells):
        a, b = offsets[c], offsets[c + 1]
        parent[a] = -1
        idx = np.arange(a + 1, b)
        prev = idx - 1
        rnd = a + np.floor(r[a + 1:b] * (idx - a)).astype(np.int64)
        parent[a + 1:b] = np.where(u[a + 1:b] < branch_p, rnd, prev)
    ga = s.loguniform(n, 0.5, 50.0)
    gb = ga * s.uniform(n, 0.5, 2.0)
    ga[offsets[:-1]] = 0.0
    gb[offsets[:-1]] = 0.0
    return dict(parent=parent, ga=ga, gb=gb, offsets=offsets, n_nodes=n)
