"""Multi-rank layout of the benchmark: the hot path shards without any
exchange (compartments are independent), so every rank simulates its own
network of the same size (weak scaling).  The only collectives are a
barrier around the timed region and a max-reduction of the elapsed time.
"""
from __future__ import annotations

import os


def rank_info():
    """(rank, world_size, local_rank) from the torchrun environment."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def network_seed(base_seed: int, rank: int) -> int:
    """Seed of rank's own network (distinct per rank, same for every run)."""
    return base_seed + 1000 * rank


def aggregate(ms_local: float, instance_steps_local: float, dist=None, device=None):
    """Whole-job throughput: the instance-steps of all ranks over the slowest
    rank's time.  Returns (value, ms_max)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return instance_steps_local / (ms_local * 1e-3), ms_local
    import torch
    t = torch.tensor([ms_local, instance_steps_local], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    mx = t[:1].clone()
    dist.all_reduce(mx, op=dist.ReduceOp.MAX)
    tot = t[1:].clone()
    dist.all_reduce(tot, op=dist.ReduceOp.SUM)
    return float(tot.item()) / (float(mx.item()) * 1e-3), float(mx.item())
