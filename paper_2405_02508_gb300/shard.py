"""Data-parallel sharding over ranks, one process per GPU.

Views of a mesh and the meshes of an uneven batch are independent units of the path: a rank renders and
differentiates its own units and never reads another rank's data.

* Independent units (weak scaling): every rank gets the same amount of work as a single GPU would (its own 32
  views; its LPT share of a batch of ``world x n_items`` meshes); the data path has no collective, the ranks
  meet only at the timing barrier and at the max-reduction of the measured step time, and the whole-job
  throughput is the units of all ranks over the slowest rank's time.
* One mesh seen by many views (strong scaling): the views are split over the ranks (``split_views``), each rank
  computes the world-space vertex gradient of its own views, and one sum over the ranks (``sum_over_ranks``,
  an all-reduce of the [V, 3] gradient, 786 KB for the head mesh) gives every rank the gradient of all views:
  the sum over views is the only coupling of the path (the edge and interior terms are local to each view's
  pixels, Sec. 4.1).
"""
from __future__ import annotations

import heapq
import os

import numpy as np


def env_ranks() -> tuple[int, int, int]:
    """(world size, rank, local rank) from the launcher's environment (1, 0, 0 when run directly)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def item_cost(T: int, H: int, W: int) -> float:
    """Cost model of one item: triangle setup and binning scale with T, raster / shade / backward with H*W."""
    return float(T) + float(H) * float(W)


def lpt_assign(costs, world: int) -> list[list[int]]:
    """Greedy longest-processing-time assignment of units to ``world`` ranks.

    Units are taken in decreasing cost (ties: lower index first) and each goes to the currently least-loaded
    rank (ties: lower rank).  The makespan is at most (4/3 - 1/(3 world)) times the optimum (Graham's bound).
    Returns, per rank, its unit indices in increasing order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    heap = [(0.0, r) for r in range(world)]
    out: list[list[int]] = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(o) for o in out]


def loads(costs, shards) -> list[float]:
    costs = np.asarray(costs, dtype=np.float64)
    return [float(costs[s].sum()) if len(s) else 0.0 for s in shards]


def view_seed(base: int, rank: int) -> int:
    """Camera seed of a rank's own batch of views (weak scaling: distinct views per rank)."""
    return base + rank


def max_over_ranks(value: float, device=None) -> float:
    """The maximum of ``value`` over all ranks (the step time of the slowest rank); identity without a
    process group."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier() -> None:
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()


def split_views(n_views: int, world: int) -> list[list[int]]:
    """Contiguous split of a mesh's views over ``world`` ranks; shard sizes differ by at most one, the first
    ``n_views % world`` ranks taking the larger ones."""
    if world < 1:
        raise ValueError("world must be >= 1")
    q, r = divmod(n_views, world)
    out, start = [], 0
    for k in range(world):
        size = q + (1 if k < r else 0)
        out.append(list(range(start, start + size)))
        start += size
    return out


def sum_over_ranks(t):
    """Sums tensor ``t`` over all ranks in place (an all-reduce; NCCL on GPU tensors, gloo on CPU ones) and
    returns it; identity without a process group."""
    import torch.distributed as dist

    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
