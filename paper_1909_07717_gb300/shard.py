"""Host logic of the state-sharded multi-GPU path (no data-path collective).

States are independent, so each rank searches its own batch; the only
cross-rank traffic is the barrier around the timed region and one max
reduction of the elapsed time.  Rank 0 keeps the workload's own seed, the
other ranks draw from rank-derived seeds, so no two ranks repeat work.
"""
from __future__ import annotations


def rank_seed(base_seed: int, rank: int) -> int:
    """Seed of the states rank ``rank`` searches."""
    return base_seed if rank == 0 else 1000 + rank


def max_over_ranks(value: float, dist=None, device="cpu") -> float:
    """The largest ``value`` over all ranks (the job's elapsed time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: int, world: int, steps: int, max_ms: float):
    """Whole-job throughput: every rank's units over the slowest rank's time."""
    return world * units_per_rank * steps / (max_ms / 1e3)
