"""The N>1 path of the benchmark on CPU: two gloo ranks, each running its
own network shard through the FP64 oracle (the GPU ranks run the same
shards through the library), aggregated exactly as bench.py does."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import oracle as orc
    from paper_1905_02241_b300 import workloads as W
    from paper_1905_02241_b300.sharding import aggregate, network_seed, rank_info
    r, w, _ = rank_info()
    assert (r, w) == (rank, world)
    wl = W.cortical_mix(300, seed=network_seed(2, r))
    st = [orc.mech_init(m["type"], m["params"], m["node_index"], wl["v0"])
          for m in wl["mechs"]]
    v, _, _, _ = orc.step(wl["mechs"], st, wl["v0"], 300, 0.025, nsteps=5)
    ninst = sum(m["node_index"].size for m in wl["mechs"])
    ms_local = 10.0 * (rank + 1)                   # a slower second rank
    dist.barrier()
    value, ms = aggregate(ms_local, float(ninst) * 5, dist)
    out[rank] = (value, ms, ninst, float(v.sum()))
    dist.destroy_process_group()


def test_two_gloo_ranks_weak_scaling():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    (v0, ms0, n0, s0), (v1, ms1, n1, s1) = out[0], out[1]
    assert ms0 == ms1 == 20.0                      # max over ranks
    assert v0 == v1 == pytest.approx((n0 + n1) * 5 / 20e-3)
    assert n0 != n1 and s0 != s1                   # each rank its own network


def test_single_rank_aggregate_is_local():
    from paper_1905_02241_b300.sharding import aggregate
    assert aggregate(4.0, 8.0) == (2000.0, 4.0)
    np.testing.assert_equal(aggregate(1.0, 1.0)[1], 1.0)
