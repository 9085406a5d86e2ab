"""Sharding the domains of one problem across ranks (one process per GPU).

Domains are independent through every step of the method (each sub-box or branch domain carries its
own Taylor model, slopes and split multipliers), so a rank bounds a contiguous block of them with no
data-path collective.  The only exchange is the final one: the reachable-set hull over all domains
(a9) is the elementwise min/max of the ranks' hulls, and the tube objective V is a sum.
"""
from typing import Tuple

import numpy as np
import torch
import torch.distributed as dist


def shard_range(D: int, rank: int, world: int) -> Tuple[int, int]:
    """[start, stop) of rank's block: sizes differ by at most one, earlier ranks take the extra."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside world of {world}")
    base, extra = divmod(int(D), world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_problem(prob, rank: int, world: int):
    """The problem restricted to this rank's domains (splits and multipliers travel with them)."""
    start, stop = shard_range(prob.D, rank, world)
    return prob.subset(np.arange(start, stop))


def merge_hull(hull_lo: torch.Tensor, hull_hi: torch.Tensor, group=None):
    """In place: hull over every rank's domains.  A rank without feasible domains passes +inf/-inf."""
    dist.all_reduce(hull_lo, op=dist.ReduceOp.MIN, group=group)
    dist.all_reduce(hull_hi, op=dist.ReduceOp.MAX, group=group)
    return hull_lo, hull_hi


def merge_objective(V_sum: torch.Tensor, group=None) -> torch.Tensor:
    """In place: the tube objective summed over every rank's domains."""
    dist.all_reduce(V_sum, op=dist.ReduceOp.SUM, group=group)
    return V_sum
