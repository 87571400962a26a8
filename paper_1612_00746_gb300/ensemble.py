"""Host-side logic for running an ensemble over several processes (one GPU each).

Realizations are independent (the paper's "embarrassingly parallel" problem,
Sec. 1), so ranks hold disjoint realization ids and never exchange states.
The only exchange is the last step of the ensemble average of Sec. 2
(<rho> = (1/R) sum_i |Psi_i><Psi_i|, reduced to P(x)): every rank averages its
own realizations on the GPU and the ranks combine their means weighted by
their realization counts, in FP64.
"""
from __future__ import annotations

from typing import List

import torch
import torch.distributed as dist


def shard_realizations(total: int, world: int, rank: int) -> List[int]:
    """Contiguous block of realization ids of one rank (sizes differ by at most 1)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def combine_means(P_mean: torch.Tensor, counts: torch.Tensor) -> torch.Tensor:
    """Ensemble mean over all ranks from per-rank means.

    P_mean: [..., width] FP64 mean of this rank's realizations per output
    column; counts: [width] FP64 number of realizations behind each column on
    this rank (0 where the rank has none).  Returns sum_k c_k P_k / sum_k c_k
    (columns with no realization anywhere are 0).
    """
    num = P_mean.to(torch.float64) * counts.to(torch.float64)
    den = counts.to(torch.float64).clone()
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(num, op=dist.ReduceOp.SUM)
        dist.all_reduce(den, op=dist.ReduceOp.SUM)
    return torch.where(den > 0, num / torch.clamp(den, min=1.0), torch.zeros_like(num))


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value of a scalar over all ranks (timing: the slowest rank)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
