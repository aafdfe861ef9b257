"""Replicas across GPUs: the repair of one field does not shard in one exchange (every
round would need a halo exchange), so N GPUs run N independent compressions, one
field each, with no collective on the data path.  This module holds the host logic
of that mode: each rank's field seed, the slowest rank's step time, and the
whole-job throughput (weak scaling: per-GPU work is fixed as N grows)."""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the field a rank compresses (every rank has its own field)."""
    return base_seed + rank


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The largest value over all ranks (the slowest rank's time); `dist` is
    torch.distributed (any backend) or None for a single process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_gbs(bytes_per_rank: int, world: int, ms_step_max: float) -> float:
    """Uncompressed bytes all ranks processed per step over the slowest rank's step time."""
    if ms_step_max <= 0:
        raise ValueError("step time must be positive")
    return world * bytes_per_rank / (ms_step_max * 1e-3) / 1e9
