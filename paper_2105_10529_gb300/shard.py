"""Event sharding across ranks (one process per GPU) for the VEGAS passes.

Events are independent and the Philox stream is indexed by the event number,
so rank r of a world of W ranks evaluates events [r N, (r + 1) N) of the same
counter space that a single device would evaluate as [0, W N).  Each rank's
pass normalises its weights by its own N; after the pass sums are added over
the ranks, rescaling gives exactly the sums of the single W N-event pass
(up to the order of the additions):

    sum_e w_e / (W N)        = (1 / W)   * sum_r [sum_{e in r} w_e / N]
    sum_e (w_e / (W N))^2    = (1 / W^2) * sum_r [sum_{e in r} (w_e / N)^2]

and the same 1 / W^2 for the per-bin sums of squares.  Every rank then
refines the same grid from the same sums, so the grids stay identical
without broadcasting them.  The only exchange is one all-reduce of
2 + D n_bins doubles per iteration.
"""
from __future__ import annotations

from typing import Tuple


def event_range(n_per_rank: int, rank: int) -> Tuple[int, int]:
    """(first event, number of events) of this rank."""
    if n_per_rank < 1 or rank < 0:
        raise ValueError("event_range: n_per_rank >= 1 and rank >= 0")
    return rank * n_per_rank, n_per_rank


def rescale_reduced_sums(sums, world: int):
    """In place: turn the rank-sum of per-rank pass sums [2 + D n_bins]
    (index 0 the weight sum, the rest sums of squares) into the sums of one
    pass over all ranks' events."""
    if world < 1:
        raise ValueError("world >= 1")
    sums[0] = sums[0] / world
    sums[1:] = sums[1:] / (world * world)
    return sums


def allreduce_pass_sums(sums, world: int, group=None):
    """All-reduce (sum) a pass-sum tensor over the process group and rescale it."""
    import torch.distributed as dist
    if world > 1:
        dist.all_reduce(sums, group=group)
    return rescale_reduced_sums(sums, world)
