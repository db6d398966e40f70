"""Host-side logic of running the step on several GPUs as independent replicas.

The single-problem path is not split across GPUs: each rank owns whole
problems, so no data-path collective exists.  Independent scenarios (the
batched workload) are dealt round-robin over the ranks; a replicated single
problem runs once per rank.  The only collective is the timing reduction
after the timed region: the job's duration is the slowest rank's.

Everything here is plain Python over ``torch.distributed`` and runs with the
``gloo`` backend on CPU as well as with NCCL on GPUs.
"""
from __future__ import annotations

from typing import Sequence


def shard(n_problems: int, rank: int, world: int) -> list[int]:
    """Indices of the problems rank ``rank`` of ``world`` steps (round-robin).

    Every index in ``range(n_problems)`` goes to exactly one rank; the counts
    of two ranks differ by at most one.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} is outside a world of {world}")
    if n_problems < 0:
        raise ValueError("n_problems must be non-negative")
    return list(range(rank, n_problems, world))


def max_over_ranks(values: Sequence[float], dist=None, device=None) -> list[float]:
    """Element-wise maximum of ``values`` over all ranks (FP64 all-reduce).

    With ``dist`` None (one process) the values come back unchanged.
    ``device`` is where the reduction buffer lives: a CUDA device for NCCL,
    None (CPU) for gloo.
    """
    vals = [float(v) for v in values]
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def sum_over_ranks(values: Sequence[float], dist=None, device=None) -> list[float]:
    """Element-wise sum of ``values`` over all ranks (the units all ranks processed)."""
    vals = [float(v) for v in values]
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t.tolist()


def job_rate(units_all_ranks: float, seconds_max: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    if seconds_max <= 0.0:
        raise ValueError("the timed region must have a positive duration")
    return units_all_ranks / seconds_max
