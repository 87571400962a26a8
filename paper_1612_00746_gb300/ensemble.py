"""Host-side logic for running an ensemble over several processes (one GPU each).

Realizations are independent (the paper's "embarrassingly parallel" problem,
Sec. 1), so ranks hold disjoint realization ids and never exchange states.
The only exchanges are the last step of the ensemble average of Sec. 2
(<rho> = (1/R) sum_i |Psi_i><Psi_i|, reduced to P(x)): every rank averages its
own realizations on the GPU and the ranks combine their means weighted by
their realization counts, in FP64; and, for the gradient of a loss on that
average, one FP64 sum of the ranks' gradient sums.

A rank that stops (an exception, an exit) is reported to the others instead
of leaving them blocked: collectives run under the process group's timeout
and raise RankFailure, and Heartbeat lets the ranks check, before each step's
launches, that all of them reached the previous one.
"""
from __future__ import annotations

import datetime
from typing import List, Optional, Sequence

import numpy as np
import torch
import torch.distributed as dist


class RankFailure(RuntimeError):
    """Another rank did not take part in an exchange within the timeout."""


def _multi() -> bool:
    return dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1


def _all_reduce(t: torch.Tensor, op) -> None:
    try:
        dist.all_reduce(t, op=op)
    except RuntimeError as e:   # gloo / NCCL timeouts and broken connections
        raise RankFailure(f"rank {dist.get_rank()}: a collective did not complete ({e})") from e


def shard_realizations(total: int, world: int, rank: int) -> List[int]:
    """Contiguous block of realization ids of one rank (sizes differ by at most 1)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    base, extra = divmod(total, world)
    start = rank * base + min(rank, extra)
    return list(range(start, start + base + (1 if rank < extra else 0)))


def shard_by_cost(sizes: Sequence[int], m: int, world: int, rank: int) -> List[int]:
    """Realization ids of one rank for a ragged batch, balanced by cost.

    The work of realization r is proportional to its N_r^m amplitudes.  The
    realizations are taken largest first (ties by id) and each goes to the
    rank with the least work so far (ties to the lowest rank): the largest
    rank load exceeds the mean by at most one realization's cost.  Returns
    the rank's ids in ascending order; every rank computes the same split.
    """
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad world/rank")
    cost = np.asarray(sizes, dtype=np.float64) ** int(m)
    order = sorted(range(len(cost)), key=lambda r: (-cost[r], r))
    load = np.zeros(world)
    owner = np.empty(len(cost), dtype=np.int64)
    for r in order:
        k = int(np.argmin(load))
        owner[r] = k
        load[k] += cost[r]
    return [int(r) for r in np.flatnonzero(owner == rank)]


def combine_means(P_mean: torch.Tensor, counts: torch.Tensor) -> torch.Tensor:
    """Ensemble mean over all ranks from per-rank means.

    P_mean: [..., width] FP64 mean of this rank's realizations per output
    column; counts: [width] FP64 number of realizations behind each column on
    this rank (0 where the rank has none).  Returns sum_k c_k P_k / sum_k c_k
    (columns with no realization anywhere are 0).  RankFailure if a rank
    does not join within the process group's timeout.
    """
    num = P_mean.to(torch.float64) * counts.to(torch.float64)
    den = counts.to(torch.float64).clone()
    if _multi():
        _all_reduce(num, dist.ReduceOp.SUM)
        _all_reduce(den, dist.ReduceOp.SUM)
    return torch.where(den > 0, num / torch.clamp(den, min=1.0), torch.zeros_like(num))


def sum_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """FP64 sum of a tensor over all ranks (a copy; RankFailure on a timeout)."""
    out = t.to(torch.float64).clone()
    if _multi():
        _all_reduce(out, dist.ReduceOp.SUM)
    return out


def max_over_ranks(value: float, device="cpu") -> float:
    """Largest value of a scalar over all ranks (timing: the slowest rank)."""
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    if _multi():
        _all_reduce(t, dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- gradients
# The loss sum_x (Pbar(x, T) - P*(x))^2 is a function of the mean over ALL
# realizations, so a rank cannot take its gradient from its own mean alone.
# With Pbar the global mean, the gradient with respect to a parameter shared
# by group g is sum_r 2 (Pbar - P*) . dP_r/dtheta / R_g over every rank's
# realizations r.  A rank's adjoint (ctqw_adjoint_grad) forms
# 2 (Pbar_k - target) . dP_r/dtheta / R_g,k from its own mean Pbar_k and its
# own count R_g,k; given target = P* + Pbar_k - Pbar its difference is the
# global one, and the factor R_g,k / R_g turns its count into the global one.
# The ranks' scaled sums then add up (one FP64 all-reduce) to the gradient.

def adjoint_target(P_target: torch.Tensor, P_local: torch.Tensor, P_global: torch.Tensor) -> torch.Tensor:
    """Target to pass to a rank's adjoint so that its loss difference
    Pbar_local - target equals the global Pbar - P_target."""
    return P_target.to(torch.float64) + P_local.to(torch.float64) - P_global.to(torch.float64)


def combine_gradients(grad_sum: torch.Tensor, counts_local: torch.Tensor,
                      counts_global: torch.Tensor) -> torch.Tensor:
    """Global gradient from the ranks' gradients with respect to the group means.

    grad_sum: [width] FP64, this rank's sums over its realizations of each
    group (ctqw_adjoint_grad's grad_*_mean, computed with adjoint_target);
    counts_local / counts_global: [width] realizations behind each column on
    this rank / on all ranks.  Returns sum_k (R_g,k / R_g) grad_sum_k.
    """
    w = torch.where(counts_global > 0, counts_local.to(torch.float64) / torch.clamp(counts_global.to(torch.float64), min=1.0),
                    torch.zeros_like(counts_global, dtype=torch.float64))
    return sum_over_ranks(grad_sum.to(torch.float64) * w)


def global_loss(P_global: torch.Tensor, P_target: torch.Tensor) -> float:
    """sum_x (Pbar(x) - P*(x))^2 of the global mean (the same on every rank)."""
    return float(torch.sum((P_global.to(torch.float64) - P_target.to(torch.float64)) ** 2).item())


# ---------------------------------------------------------------- liveness
class Heartbeat:
    """Per-step liveness of the ranks through the process group's store.

    beat(step) marks this rank as having reached `step`; check(step) waits up
    to `timeout` for every other rank to have marked it, and raises
    RankFailure naming the ranks that did not.  Call beat then check before a
    step's launches, so that a rank that stopped between steps is found on
    the host, with no kernel or collective of this rank in flight.
    """

    def __init__(self, timeout_s: float = 10.0, store: Optional[dist.Store] = None,
                 rank: Optional[int] = None, world: Optional[int] = None, prefix: str = "ctqw/alive"):
        self.store = store if store is not None else dist.distributed_c10d._get_default_store()
        self.rank = dist.get_rank() if rank is None else int(rank)
        self.world = dist.get_world_size() if world is None else int(world)
        self.timeout = datetime.timedelta(seconds=float(timeout_s))
        self.prefix = prefix

    def _key(self, step: int, rank: int) -> str:
        return f"{self.prefix}/{int(step)}/{int(rank)}"

    def beat(self, step: int) -> None:
        self.store.set(self._key(step, self.rank), "1")

    def check(self, step: int) -> None:
        missing = []
        for k in range(self.world):
            if k == self.rank:
                continue
            try:
                self.store.wait([self._key(step, k)], self.timeout)
            except Exception:   # the store raises on timeout (type differs by version)
                missing.append(k)
        if missing:
            raise RankFailure(f"rank {self.rank}: rank(s) {missing} did not reach step {step} "
                              f"within {self.timeout.total_seconds():g} s")
