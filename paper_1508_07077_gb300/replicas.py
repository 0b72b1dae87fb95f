"""Sharding of independent replicas over ranks (one process per GPU).

The implicit-depletant sampler parallelises over independent systems with no
exchange between them, so a multi-GPU job is a set of replica batches, one per
rank, and there is no collective on the data path.  Rank r of a world of W
ranks owns the replicas r * per_rank ... (r + 1) * per_rank - 1; the replica
index keys the counter-based random streams (Philox key = (seed_lo, seed_hi
XOR replica)), so every rank samples its own reproducible trajectories and
the set of trajectories does not depend on how many ranks share the work
(weak scaling).  Throughput is the units all ranks processed over the slowest
rank's time: a sum and a maximum over ranks, taken with torch.distributed
(NCCL on GPUs, gloo on CPUs) when a process group is initialised.
"""
from __future__ import annotations

import os


def world():
    """(world size, rank, local rank) from the launcher's environment."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def replica_ids(per_rank: int, rank: int) -> list[int]:
    """Replica indices owned by `rank` when every rank runs `per_rank`."""
    if per_rank < 1 or rank < 0:
        raise ValueError("per_rank must be >= 1 and rank >= 0")
    return [rank * per_rank + k for k in range(per_rank)]


def _reduce(values, op, device):
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=op)
    return [float(x) for x in t.cpu()]


def reduce_max(values, device="cpu"):
    """Element-wise maximum over ranks (identity without a process group)."""
    import torch.distributed as dist
    return _reduce(values, dist.ReduceOp.MAX, device)


def reduce_sum(values, device="cpu"):
    """Element-wise sum over ranks (identity without a process group)."""
    import torch.distributed as dist
    return _reduce(values, dist.ReduceOp.SUM, device)


def world_rate(local_units: float, local_seconds: float, device="cpu") -> float:
    """Whole-job throughput: units of every rank over the slowest rank's time."""
    units = reduce_sum([local_units], device)[0]
    seconds = reduce_max([local_seconds], device)[0]
    return units / seconds
