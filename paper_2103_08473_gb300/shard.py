"""Host-side sharding of independent systems across GPUs (one process per GPU).

A batch of independent CCSD systems needs no exchange while it is solved: rank r solves the
systems assigned to it, and only the per-system results travel, once, at the end. This
module holds the two host steps of that split, used by the batched benchmark:

* ``partition``: systems to ranks, balanced by an estimate of their cost (the ladder's
  o^2 v^4 by default), by the longest-processing-time rule: systems in order of decreasing
  cost, each to the rank with the least total so far (ties: the lower rank). Every system
  goes to exactly one rank; within a rank the systems keep their batch order.
* ``gather_results``: each rank's per-system rows (a fixed number of float64 values per
  system) into one (nsys, width) array on every rank, by a single all_gather of fixed-size
  arrays: each rank sends an (nsys, width + 1) array whose last column flags the rows it
  owns, and each row is taken from its owner.
"""
from __future__ import annotations

import numpy as np


def ladder_cost(o: int, v: int) -> float:
    """Relative cost of one system: the particle-particle ladder's o^2 v^4."""
    return float(o) ** 2 * float(v) ** 4


def partition(costs, world: int):
    """Assign system k (cost costs[k]) to a rank; returns a list of `world` index lists."""
    if world < 1:
        raise ValueError("world must be >= 1")
    costs = [float(c) for c in costs]
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for k in sorted(range(len(costs)), key=lambda k: (-costs[k], k)):
        r = min(range(world), key=lambda r: (load[r], r))
        parts[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in parts]


def gather_results(rows: dict, nsys: int, width: int):
    """rows: {system index: sequence of `width` floats} of this rank. Returns the (nsys, width)
    float64 array of every system's row, identical on every rank (torch.distributed must be
    initialised when world > 1; rows of systems no rank owns stay NaN)."""
    import torch
    import torch.distributed as dist

    mine = np.full((nsys, width + 1), np.nan)
    mine[:, width] = 0.0
    for k, vals in rows.items():
        mine[k, :width] = np.asarray(vals, dtype=np.float64)
        mine[k, width] = 1.0
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return mine[:, :width].copy()
    backend = dist.get_backend()
    device = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.from_numpy(mine).to(device)
    parts = [torch.empty_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(parts, t)
    out = np.full((nsys, width), np.nan)
    owners = np.zeros(nsys, dtype=np.int64)
    for p in parts:
        a = p.cpu().numpy()
        own = a[:, width] == 1.0
        out[own] = a[own, :width]
        owners += own
    if np.any(owners > 1):
        raise RuntimeError("a system was solved on more than one rank")
    return out
