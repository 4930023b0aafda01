"""Host logic of the multi-GPU benchmark: independent replicas.

Frame pairs are independent, so N GPUs run N replicas, each on its own pairs,
with no collective on the data path.  The only cross-rank operations are a
barrier around the timed region and a max-reduction of the elapsed time;
whole-job throughput is every rank's pixels divided by the slowest rank's
time (weak scaling).
"""

from __future__ import annotations


def rank_pair_indices(rank: int, world: int, per_rank: int):
    """Pair indices of one rank: disjoint across ranks, `per_rank` each."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return list(range(rank * per_rank, (rank + 1) * per_rank))


def max_over_ranks(value: float, device=None) -> float:
    """Max of `value` over all ranks (identity without a process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64,
                     device=device if device is not None else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds_max: float) -> float:
    """Units per second of the whole job: all ranks' units over the slowest
    rank's time."""
    return units_per_rank * world / seconds_max
