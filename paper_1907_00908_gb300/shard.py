"""Sharding of independent members (directions, b-values, geometries) across
ranks, one GPU per rank.

Members never exchange data: a rank runs its share through the library and
only results (3 doubles per member) and timings cross ranks, on the host.
There is no collective on the data path.
"""
from __future__ import annotations

import numpy as np


def assign(costs, world):
    """Longest-processing-time greedy split of member indices over ``world``
    ranks (deterministic: ties go to the lower rank, members in input order)."""
    costs = np.asarray(costs, dtype=np.float64)
    order = sorted(range(len(costs)), key=lambda i: (-costs[i], i))
    load = [0.0] * world
    out = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        out[r].append(i)
        load[r] += costs[i]
    return [sorted(x) for x in out]


def gather_results(local_idx, local_vals, n_total, dist=None):
    """Assemble per-member result rows from every rank (host all-gather)."""
    rows = list(zip(local_idx, [np.asarray(v).tolist() for v in local_vals]))
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        parts = [None] * dist.get_world_size()
        dist.all_gather_object(parts, rows)
        rows = [r for p in parts for r in p]
    out = [None] * n_total
    for i, v in rows:
        out[i] = v
    if any(v is None for v in out):
        raise RuntimeError("a member has no result")
    return np.asarray(out)


def max_over_ranks(value, dist=None, device=None):
    """Maximum of a per-rank float (timings: the slowest rank sets the time)."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())
