"""Series sharding across GPUs (one process per GPU).

Independent series (or hyperparameter sets) need no exchange: each rank takes
a longest-processing-time share of the series, computes them on its own GPU,
and per-series rows are gathered only where the caller wants them in one
place.  There is no collective on the data path.
"""
from __future__ import annotations

import numpy as np


def lpt_shards(counts, world: int):
    """Assign series (weights ``counts``, e.g. measurements) to ``world``
    ranks by the longest-processing-time rule; returns sorted index lists."""
    counts = np.asarray(counts)
    order = np.argsort(-counts, kind="stable")
    loads = np.zeros(world)
    parts = [[] for _ in range(world)]
    for i in order:
        r = int(np.argmin(loads))
        parts[r].append(int(i))
        loads[r] += counts[i]
    return [sorted(p) for p in parts]


def gather_rows(local_rows, local_idx, n_total: int, group=None):
    """All-gather per-series result rows computed on each rank into the
    global series order (every rank receives the full array)."""
    import torch.distributed as dist
    local_rows = np.asarray(local_rows)
    world = dist.get_world_size(group)
    got = [None] * world
    dist.all_gather_object(got, (list(local_idx), local_rows), group=group)
    shape = (n_total,) + local_rows.shape[1:]
    out = np.zeros(shape, dtype=local_rows.dtype)
    seen = np.zeros(n_total, bool)
    for idx, rows in got:
        out[idx] = rows
        seen[idx] = True
    if not seen.all():
        raise RuntimeError("sharded rows do not cover every series")
    return out
