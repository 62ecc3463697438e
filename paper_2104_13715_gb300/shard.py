"""Host logic of the multi-GPU forms: one process per GPU, no collective on
the data path.

The fit shards naturally (the method has no exchange step between
independent image pairs):

* independent pairs: each rank fits its own pairs; a batch of pairs is split
  across ranks by estimated cost (longest-processing-time first), and the
  ranks meet only to combine timings and counts;
* one large image (not run on a GPU here: every call has one GPU): the valid
  region splits into row bands, each band holding its rows plus the (m - 1)
  reference rows below them that its pixels read; the loss and gradient are
  sums over pixels (Eq. 8), so the bands' partial sums add up to the whole,
  and an evaluation would need one all-reduce of m^2 + 5 float64 values.

Everything here runs with the gloo backend on CPU as well as with NCCL.
"""
from __future__ import annotations

import heapq
import os
from typing import List, Sequence, Tuple


def rank_env() -> Tuple[int, int, int]:
    """(rank, world size, local rank) from the torchrun environment."""
    g = lambda k, d: int(os.environ.get(k, d))
    return g("RANK", 0), g("WORLD_SIZE", 1), g("LOCAL_RANK", 0)


def partition_by_cost(costs: Sequence[float], world: int) -> List[List[int]]:
    """Split unit indices over `world` ranks so the largest per-rank cost is
    small: units in decreasing cost, each to the currently lightest rank
    (ties to the lower rank).  Every index appears exactly once; each rank's
    list is in increasing index order."""
    if world < 1:
        raise ValueError("world must be >= 1")
    heap = [(0.0, r) for r in range(world)]
    out: List[List[int]] = [[] for _ in range(world)]
    for i in sorted(range(len(costs)), key=lambda k: (-float(costs[k]), k)):
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + float(costs[i]), r))
    return [sorted(o) for o in out]


def pair_cost(side_y: int, side_x: int, m: int) -> float:
    """Work of one evaluation of a pair: 2 m^2 FMA per valid pixel."""
    h = m // 2
    return float(max(side_y - 2 * h, 0) * max(side_x - 2 * h, 0) * m * m)


def band_partition(H: int, m: int, world: int) -> List[Tuple[int, int]]:
    """Row bands of the valid region for `world` ranks: band r is valid rows
    [v0, v1) (valid-region coordinates, as even as possible; empty bands when
    world exceeds the valid rows) and needs image rows [v0, v1 + m - 1)."""
    nv = H - 2 * (m // 2)
    if nv < 0 or world < 1:
        raise ValueError("no valid region or bad world size")
    base, extra = divmod(nv, world)
    out, v0 = [], 0
    for r in range(world):
        v1 = v0 + base + (1 if r < extra else 0)
        out.append((v0, v1))
        v0 = v1
    return out


def band_rows(v0: int, v1: int, m: int) -> slice:
    """Image rows a band of valid rows [v0, v1) reads (its (m - 1)-row halo included)."""
    return slice(v0, v1 + m - 1)


def reduce_max_sum(ms: float, units: float, device=None) -> Tuple[float, float]:
    """Max over ranks of the timed milliseconds and sum of the units processed
    (identity without an initialised process group)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(ms), float(units)
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())
