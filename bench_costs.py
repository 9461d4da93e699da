"""Algorithmic operation counts behind the roofline figures of bench.py.

Every path of the library is bound by one arithmetic unit (HBM stays idle:
compartments are staged in shared memory for a whole window, and the kinetic
and surrogate kernels read and write each state once per step).  A count
here is the number of instructions a minimal implementation of the method
issues on that unit per instance-step; the reported fraction is
count x (instance-steps/s) / (measured peak of the unit).

FP64 paths (plain FP64 forms): FP64 pipe instructions.  add/sub/mul/fma 1;
exp, reciprocal and division at the cost of the routines this design uses
(`DESIGN`: exp 2 -- a 2048-entry table, r1 = x - n L1 and T + T p on the
FP64 pipe, n, the rest of the reduction and the degree-3 polynomial formed
in single precision and widened by integer operations; reciprocal 2 -- a
seed good to 2^-45 formed in single precision, then e = 1 - x y, y + y e;
division 2 -- a quotient good to 2^-44 formed in single precision, then
r = x - y q, q + r y0).  Moving work off the FP64 pipe lowers these counts,
so the fraction measures how fully the kernel uses the FP64 pipe for the
work the design leaves there.  `ALL_FP64` prices the same routines written
entirely in FP64 arithmetic (exp 8: two for n, two for the two-part
reduction, three for the degree-3 polynomial, one for T (1 + p);
reciprocal 3: e = 1 - x y0, e + e^2, y0 + y0 (e + e^2) from the hardware
seed; division 6: that reciprocal, q = x r, r' = x - y q, q + r' r): a
yardstick that does not move with the design.

MIXED paths: the FP64 residue (compensated sums, rhs/d accumulation, the
residuals and refinements) on the FP64 pipe, which is their narrowest unit.
Surrogate: BF16 tensor-core flops (K and N padded to 16, as run) and the
special-function unit (tanh of the SiLU, exp2 of the rates).
"""
from __future__ import annotations

from paper_1905_02241_b300 import workloads as W

# pm: FP64 instructions to form 1 +- e^x from e^x (the design takes the
# constant part 1 +- 2^m T from integer operations and folds the rest into
# the exp's last instruction)
DESIGN = dict(exp=2, rcp=2, div=2, pm=0)
ALL_FP64 = dict(exp=8, rcp=3, div=6, pm=1)


def _rate(form: int, c) -> int:
    """One rate as numerator / denominator: u = v/k - vh/k (1 fma); EXP
    e^u: exp; SIGMOID A/(1 + e^-u): exp and 1 + e^-u; LINOID A u/(1 - e^-u):
    exp, 1 - e^-u and the multiply A u."""
    return {0: 1 + c["exp"], 1: 1 + c["exp"] + c["pm"], 2: 1 + c["exp"] + c["pm"] + 1}[form]


def _gate_tail(aform: int, bform: int, c) -> int:
    """minf and phi dt (alpha + beta) from the two rates (N = Pa Db + Pb Da,
    D = Da Db; an EXP rate's denominator is 1), then the cnexp update
    minf + (m - minf) exp(-phi dt s): exp, difference, fma."""
    if aform == 0 and bform == 0:
        comb = 1 + c["div"]
    elif bform == 0:
        comb = 1 + 2 * c["div"]
    elif aform == 0:
        comb = 2 + 2 * c["div"]
    else:
        comb = 3 + 2 * c["div"]
    return comb + c["exp"] + 2


def _node(c) -> int:
    """per node: rhs = sum(g e) - v sum(g), d += cm/dt, 1/d, v += rhs (1/d)"""
    return 1 + 1 + c["rcp"] + 1


HH_GATES = ((2, 0), (0, 1), (2, 0))   # (alpha, beta) forms of m, h, n


def fp64_ops_per_step(wl, c=DESIGN) -> float:
    """FP64 pipe instructions of one network time step (cur + v + state) of
    an isolated-compartment cnexp network (HH and generic gates)."""
    ops = _node(c) * wl["n_nodes"]
    for m in wl["mechs"]:
        p, n = m["params"], m["node_index"].size
        if m["type"] == W.TYPE_HH:
            # three gates; gna = g m^3 h and gk = g n^4 (4 multiplies each);
            # three currents summed into the node (2 each)
            per = sum(_rate(a, c) + _rate(b, c) + _gate_tail(a, b, c) for a, b in HH_GATES)
            per += 4 + 4 + 3 * 2
        elif m["type"] == W.TYPE_CNEXP:
            per, pw = 0, 0
            for g in range(int(p[0])):
                o = 6 + 9 * g
                af, bf = int(p[o + 1]), int(p[o + 5])
                per += _rate(af, c) + _rate(bf, c) + _gate_tail(af, bf, c)
                pw += int(p[o])
            per += pw + 2                    # gbar x^p, then summed into the node
        elif m["type"] == W.TYPE_KIN3:
            per = kin3_fp64_ops(c)
        elif m["type"] == W.TYPE_CACUM:
            per = cacum_fp64_ops(c)
        else:
            raise ValueError(f"no FP64 count for mechanism type {m['type']}")
        ops += per * n
    return float(ops)


# ------------------------------------------------------------ kinetic schemes

KIN9_EDGES = 12
KIN9_BAND = 3        # states 3a + b on the 3x3 lattice: |i - j| <= 3


def _band_lu_counts(nst: int, band: int, c):
    """(factorisation, one solve) of the no-pivot LU restricted to the band
    |i - j| <= band: per pivot its reciprocal; per row below it inside the
    band one multiplier and one fma per band entry to its right; a solve
    takes one fma per off-diagonal band entry and one multiply per row."""
    def inb(i, j):
        return abs(i - j) <= band
    lu = 0
    for k in range(nst):
        lu += c["rcp"]
        for i in range(k + 1, nst):
            if inb(i, k):
                lu += 1 + sum(1 for j in range(k + 1, nst) if inb(k, j) and inb(i, j))
    off = sum(1 for i in range(nst) for j in range(nst) if i != j and inb(i, j))
    return lu, off + nst


def kin9_fp64_ops(updates: float = 2.0, c=DESIGN) -> float:
    """One implicit-Euler step of the 9-state scheme by Newton with the
    banded LU, `updates` Newton updates (2 for a linear scheme: the first
    is exact, the second confirms it), plus its current and the clamped
    node.  Rates dt k = exp(b v + ln(dt a)): fma + exp each (24); the
    diagonal of J accumulated from them (24 adds); per update the residual
    x - J y (9 + 24 fma), the two triangular solves and y += delta (9)."""
    lu, solve = _band_lu_counts(9, KIN9_BAND, c)
    rates = 2 * KIN9_EDGES * (1 + c["exp"])
    per_update = (9 + 2 * KIN9_EDGES) + solve + 9
    cur = 1 + 2 + 2              # g = gbar x_open, i = g (v - e), into rhs and d
    node = 1                     # d += cm/dt (v clamped)
    return rates + 2 * KIN9_EDGES + lu + updates * per_update + cur + node


def kin9_mixed_fp64_ops(updates: float) -> float:
    """FP64 residue of the mixed 9-state step (FP32 rates and LU; the
    residual's rate products and sums and J's diagonal as float pairs on the
    FP32 pipe): per update x - y (9) and y += delta (9), the current and the
    node."""
    return updates * (9 + 9) + 5 + 1


def kin3_fp64_ops(c=DESIGN) -> int:
    """3-state scheme, one step = one solve: 6 rates (multiply + exp each;
    the exponent b v is one multiply), M = I - dt A (6 multiplies for the
    off-diagonals, 6 fma for the diagonal), the written-out 3x3 elimination
    (three pivot reciprocals, 3 multipliers, 5 updates) and its solve (3 +
    3 multiply-adds, 3 multiplies); its current (g, then into the node: 3)."""
    rates = 6 * (2 + c["exp"])
    matrix = 6 + 6
    elim = 3 * c["rcp"] + 3 + 5
    solve = 3 + 3 + 3
    return rates + matrix + elim + solve + 3


def cacum_fp64_ops(c=DESIGN, updates: float = 4.0) -> float:
    """Calcium buffer: per Newton update the residual (fr = btot - y1,
    on = kf fr, off = kf y0 + kb, bind = on y0 - kb y1, f0 = src - rtau y0 -
    bind, r0 = x0 - y0 + dt f0, r1 = x1 - y1 + dt bind: 11), the Jacobian
    and its determinant (q = dt on, p = dt off, a = 1 + dt (on + 1/tau),
    d = 1 + p, det = a d - p q: 7) and its reciprocal, delta = adj(J) r /
    det and y += delta (8); the source term once (1)."""
    return 1 + updates * (11 + 7 + c["rcp"] + 8)


# --------------------------------------------------------------- mixed cnexp

def mixed_fp64_ops_per_step(wl) -> float:
    """FP64 residue of the mixed fused step without ion arrays: per node
    v += dv (1).  The node sums of g e and g and the update's r = X - v G,
    d = G + cm/dt and r/d run as float pairs on the FP32 pipe."""
    return float(wl["n_nodes"])


# ----------------------------------------------------------------- cable

def cable_fp64_ops_per_step(wl, parent) -> float:
    """The isolated step's count with the diagonal update (1/d, v += r/d: 3
    per node) replaced by the tree system: per non-root node its axial terms
    in its own and its parent's row (4); per node v += dv (1).  The
    elimination, the pivots' reciprocals and the substitution run in float
    pairs on the FP32 pipe (no FP64 instructions)."""
    import numpy as np
    n = wl["n_nodes"]
    nonroot = int(np.count_nonzero(np.asarray(parent) >= 0))
    iso = fp64_ops_per_step(wl)
    return iso - (DESIGN["rcp"] + 1) * n + nonroot * 4 + n


# ------------------------------------------------------------- surrogate

MLP_FLOPS = 2 * (16 * 128 + 2 * 128 * 128 + 128 * 16)          # forward, padded: 73,728
# training row: forward, the three backward products D W (K = 16, 128,
# 128) and the four weight-gradient products D^T H
TRAIN_FLOPS_PER_ROW = MLP_FLOPS + 2 * (16 * 128 + 2 * 128 * 128) + MLP_FLOPS
SUR_MUFU = 3 * 128 + 2 * KIN9_EDGES      # SiLU tanh per hidden unit, exp2 per rate


# FP64 warp instructions per step of one warp of the single-HH gate-warp
# kernel (ncu on the 4,096-node HH workload: FP64 pipe 33 % active on the
# SMs, three of whose four sub-partitions hold a gate warp, 2.24 us per
# step at 2.03 GHz and one warp instruction per 68.6 clocks -> about 30;
# the FP64 operations written in the kernel's source give 22-27 per gate
# warp; the measured count is used)
HH_WARP_FP64_PER_STEP = 30

# Warp instructions the mixed-precision fused step issues per instance-step
# (measured, not modelled: ncu smsp__inst_executed.sum of one 40-step launch
# on the 1,000,000-node cortical mix, 4,074,252,771 instructions over
# 11,548,985 instances x 40 steps), for its issue-rate roofline: an SM
# issues at most one warp instruction per cycle on each of its four
# sub-partitions.
MIXED_WARP_INSTR_PER_STEP = 4074252771 / (11548985 * 40)
ISSUE_PER_SM_PER_CYCLE = 4
