"""The algorithmic FP64 count behind bench.py's roofline, pinned per form.

The numerator of the reported roofline fraction is bench.fp64_ops_per_step:
the FP64 pipe instructions of a minimal implementation of the step.  These
tests hand-count single-gate mechanisms from the device routines (u one
fma; exp 2; a SIGMOID denominator 1 + e^-u 2; LINOID's A u 1 more; minf and
phi dt (alpha + beta) as two divisions of 2, from Pa Db, N and Da Db; the
cnexp update exp 2 + difference 1 + fma 1; per instance the conductance's
powers and 2 to add it into the node; per node 5) so that a change of the
model shows up here first.
"""
import numpy as np

import bench
from paper_1905_02241_b300 import workloads as W


def _one_gate(af, bf, power, n=1000):
    p = W.cnexp_params(1e-3, -70.0, [(power, (af, 0.1, -40.0, 10.0), (bf, 0.2, -60.0, -12.0))])
    ni = np.arange(n, dtype=np.int32)
    return dict(n_nodes=n, mechs=[dict(type=W.TYPE_CNEXP, params=p, node_index=ni)])


EXP, SIG, LIN = 0, 1, 2
# u (1) + exp (2); SIGMOID: u (1) + 1 + e^-u (2); LINOID: u (1) + A u (1) + 1 - e^-u (2)
RATE = {EXP: 3, SIG: 3, LIN: 4}
# minf and phi dt (alpha + beta) from the rates, then the cnexp update (4)
TAIL = {(EXP, EXP): 1 + 2 + 4,          # s = Pa + Pb; minf = Pa / s
        (SIG, EXP): 1 + 2 * 2 + 4,      # N = Pa + Pb Da; Pa / N; N / Da
        (LIN, EXP): 1 + 2 * 2 + 4,
        (EXP, SIG): 2 + 2 * 2 + 4,      # Pa Db; N = Pb + Pa Db; Pa Db / N; N / Db
        (EXP, LIN): 2 + 2 * 2 + 4,
        (SIG, SIG): 3 + 2 * 2 + 4,      # Pa Db, N, Da Db; two divisions
        (SIG, LIN): 3 + 2 * 2 + 4,
        (LIN, SIG): 3 + 2 * 2 + 4,
        (LIN, LIN): 3 + 2 * 2 + 4}
NODE = 5                                # r = X - v G, d += cm/dt, 1/d (2), v += r/d


def test_cost_model_matches_the_hand_count_of_every_form_pair():
    for (af, bf), tail in TAIL.items():
        for power in (1, 3):
            wl = _one_gate(af, bf, power)
            per_node = NODE + RATE[af] + RATE[bf] + tail + power + 2
            assert bench.fp64_ops_per_step(wl) == per_node * wl["n_nodes"], (af, bf, power)


def test_cost_model_of_hh():
    # gates (LINOID, EXP), (EXP, SIGMOID), (LINOID, EXP); gna m^3 h and gk n^4
    # (4 multiplies each) and three currents into the node (2 each)
    n = 100
    wl = dict(n_nodes=n, mechs=[dict(type=W.TYPE_HH, params=W.hh_params(),
                                     node_index=np.arange(n, dtype=np.int32))])
    gates = (RATE[LIN] + RATE[EXP] + TAIL[(LIN, EXP)]
             + RATE[EXP] + RATE[SIG] + TAIL[(EXP, SIG)]
             + RATE[LIN] + RATE[EXP] + TAIL[(LIN, EXP)])
    assert bench.fp64_ops_per_step(wl) == (NODE + gates + 4 + 4 + 3 * 2) * n


def test_cost_model_of_the_cortical_mix_is_in_range():
    wl = W.cortical_mix(20000, seed=2)
    per = bench.fp64_ops_per_step(wl) / bench.n_instances(wl)
    assert 25.0 < per < 35.0


# ------------------------------------------------------------------------
# The other forms' counts (bench_costs), each against a hand count.

import bench_costs as C  # noqa: E402


def test_banded_lu_of_the_lattice_scheme():
    # 9 states, band |i - j| <= 3: pivots k = 0..5 each eliminate 3 rows,
    # each row a multiplier + 3 updates (12); k = 6: 2 rows of 1 + 2 (6);
    # k = 7: 1 row of 1 + 1 (2); 9 reciprocals of 2.  A solve: one fma per
    # off-diagonal band entry (2 (8 + 7 + 6) = 42) and a multiply per row (9).
    assert C._band_lu_counts(9, 3, C.DESIGN) == (6 * 12 + 6 + 2 + 9 * 2, 42 + 9)


def test_kinetic_counts():
    # rates 24 (fma + exp 2); diagonal 24; LU 98; per update residual 9 + 24,
    # solve 51, y += delta 9; current 5; node 1
    assert C.kin9_fp64_ops(2.0) == 24 * 3 + 24 + 98 + 2 * (33 + 51 + 9) + 5 + 1
    assert C.kin9_fp64_ops(2.0, C.ALL_FP64) == 24 * 9 + 24 + (80 + 9 * 3) + 2 * (33 + 51 + 9) + 6
    # mixed: diagonal 24, per update residual 33 + update 9, current and node 6
    assert C.kin9_mixed_fp64_ops(3.0) == 3 * 18 + 6


def test_small_system_counts():
    # 3-state: 6 rates (mul, exp, mul), 12 for M, 3 reciprocals + 8, solve 9, current 3
    assert C.kin3_fp64_ops() == 6 * 4 + 12 + (3 * 2 + 8) + 9 + 3
    # buffer: source 1 + 4 updates of residual 11, Jacobian 7, reciprocal 2, update 8
    assert C.cacum_fp64_ops() == 1 + 4 * (11 + 7 + 2 + 8)


def test_all_fp64_yardstick_prices_each_routine_in_fp64():
    wl = _one_gate(SIG, LIN, 2)
    # design: SIG 3, LIN 4, tail 3 + 2*2 + 4 = 11; all-FP64: SIG 1 + 8 + 1,
    # LIN 1 + 8 + 1 + 1, tail 3 + 2*6 + 8 + 2
    assert C.fp64_ops_per_step(wl) == (NODE + 3 + 4 + 11 + 2 + 2) * wl["n_nodes"]
    all64 = (1 + 1 + 3 + 1) + 10 + 11 + (3 + 12 + 8 + 2) + 2 + 2
    assert C.fp64_ops_per_step(wl, C.ALL_FP64) == all64 * wl["n_nodes"]


def test_mixed_residue_and_cable_counts():
    n = 50
    hh = dict(n_nodes=n, mechs=[dict(type=W.TYPE_HH, params=W.hh_params(),
                                     node_index=np.arange(n, dtype=np.int32))])
    # v += dv only: the node sums and the update run as float pairs
    assert C.mixed_fp64_ops_per_step(hh) == n
    # a chain of n nodes (one root): the diagonal update's 1/d and product
    # (3 per node) give way to the tree system's FP64 part: per non-root
    # node its axial terms (4), per node v += dv (the solve runs in float
    # pairs)
    parent = np.arange(-1, n - 1)
    assert C.cable_fp64_ops_per_step(hh, parent) == (
        C.fp64_ops_per_step(hh) - 3 * n + (n - 1) * 4 + n)


def test_surrogate_flop_counts():
    assert C.MLP_FLOPS == 2 * (16 * 128 + 128 * 128 + 128 * 128 + 128 * 16) == 73728
    # backward: D4 W4 (K 16), D3 W3, D2 W2; weight gradients as the forward
    assert C.TRAIN_FLOPS_PER_ROW == 73728 + 2 * (16 * 128 + 2 * 128 * 128) + 73728
