"""Splitting a batch of slices across ranks (one process per GPU).

Slices are independent: the regulariser of Sec. II-C is 2-D, per slice, so a
batch shards by slice with no exchange in the data path.  A greedy
longest-processing-time plan on cost = nx * ny * iterations balances uneven
slices; each rank solves its share on its own GPU; the results are gathered
on rank 0.  The only collective is that gather, after the solves.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence


def lpt_plan(costs: Sequence[float], world: int) -> List[List[int]]:
    """Greedy LPT: items in decreasing cost (ties by index) each go to the
    least-loaded rank (ties by rank).  Returns, per rank, its item indices in
    increasing order.  Deterministic, so every rank computes the same plan."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(costs)), key=lambda i: (-float(costs[i]), i))
    load = [0.0] * world
    plan: List[List[int]] = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        plan[r].append(i)
        load[r] += float(costs[i])
    for p in plan:
        p.sort()
    return plan


def slice_cost(nx: int, ny: int, iters: int) -> float:
    """Work of one slice: pixels times iterations."""
    return float(nx) * float(ny) * float(iters)


def solve_sharded(items: Sequence, cost: Callable[[object], float], solve: Callable[[list], list],
                  group=None) -> Optional[list]:
    """Solve ``items`` across the ranks of ``group`` (default: the default
    process group).  Rank r calls ``solve`` on its LPT share (a list of
    items, in item order) and must get one result per item back.  Rank 0
    returns the results of all items in item order; other ranks return None.
    """
    import torch.distributed as dist

    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    plan = lpt_plan([cost(x) for x in items], world)
    mine = plan[rank]
    res = list(solve([items[i] for i in mine])) if mine else []
    if len(res) != len(mine):
        raise RuntimeError(f"solve returned {len(res)} results for {len(mine)} items")
    gathered = [None] * world if rank == 0 else None
    dist.gather_object(list(zip(mine, res)), gathered, dst=0, group=group)
    if rank != 0:
        return None
    out = [None] * len(items)
    for part in gathered:
        for i, r in part:
            out[i] = r
    return out
