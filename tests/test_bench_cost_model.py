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
    assert 25.0 < per < 35.0   # 29.4 on the 1M-node mix; the kernel executes 33.0
