"""Weak-scaling shard logic of the Monte Carlo path (one process per GPU).

Trajectories are independent (Sec. 2: each is a separate noisy run of the
circuit), so N ranks split them with no data-path collective: rank k runs
trajectory counters [k T, (k+1) T) and, because the noise of a trajectory is
a pure function of (key, counter, gate) through Philox, the union over ranks
is exactly the run of N T trajectories on one device.  The only collectives
are on the host side of the measurement: a barrier around the timed region,
the maximum of the ranks' times, and (for checks) a gather of results.
"""
from __future__ import annotations

from typing import Optional, Tuple

import numpy as np


def trajectory_range(rank: int, per_rank: int) -> Tuple[int, int]:
    """First and one-past-last trajectory counter of a rank."""
    if rank < 0 or per_rank < 1:
        raise ValueError("rank must be >= 0 and per_rank >= 1")
    return rank * per_rank, (rank + 1) * per_rank


def max_over_ranks(value: float, dist=None, device: Optional[str] = None) -> float:
    """The largest of the ranks' values (the job's time is its slowest rank's)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_to_rank0(values: np.ndarray, dist=None, device: Optional[str] = None) -> Optional[np.ndarray]:
    """Concatenate every rank's equally sized float64 array on rank 0 (None elsewhere)."""
    values = np.ascontiguousarray(values, dtype=np.float64)
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return values
    import torch
    world = dist.get_world_size()
    t = torch.from_numpy(values).to(device) if device else torch.from_numpy(values)
    parts = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(parts, t)
    if dist.get_rank() != 0:
        return None
    return np.concatenate([p.cpu().numpy() for p in parts])


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job rate: the units all ranks processed over the slowest rank's time."""
    if seconds <= 0:
        raise ValueError("time must be positive")
    return units_per_rank * world / seconds
