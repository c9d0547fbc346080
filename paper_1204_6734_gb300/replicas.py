"""Multi-GPU runs as independent replicas (one lattice per rank, no data-path
collective): what each rank simulates and how the ranks' timings combine.

The method has no exchange between independent lattices, so N GPUs run N
replicas -- each rank its own lattice with its own noise stream (replica id =
rank, seed offset by rank) -- and meet only at the barriers around a timed
region. Works with any torch.distributed backend (NCCL on GPUs, gloo on CPU).
"""
from __future__ import annotations

import copy

SEED_STRIDE = 7919


def rank_params(p, rank: int):
    """The lattice rank `rank` simulates: p with its own Philox stream (third
    counter word = rank, key offset by SEED_STRIDE * rank)."""
    q = copy.copy(p)
    q.replica = int(rank)
    q.seed = int(p.seed) + SEED_STRIDE * int(rank)
    return q


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Units of all ranks per second of the slowest rank (weak scaling)."""
    return units_per_rank * world / seconds
