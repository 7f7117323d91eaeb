"""Sharding across GPUs (one process per GPU).

Independent series (or hyperparameter sets) need no exchange: each rank takes
a longest-processing-time share of the series, computes them on its own GPU,
and per-series rows are gathered only where the caller wants them in one
place.  There is no collective on the data path.

A single long series is split in time instead (Section 3.2.5, the
parallel-in-time filter, across devices): every rank builds the same
one-series model, takes a contiguous range of its chunks and forms that
range's element (gp_ss_span_element, FP64); one all-gather exchanges the
elements (a few hundred bytes per rank and parameter row) and every rank folds
them in time order into the series' log-likelihood (gp_ss_span_loglik).
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


def span_chunk_ranges(n_chunks: int, world: int):
    """Contiguous chunk ranges [c0, c1) of a one-series model for ``world``
    ranks, balanced (the chunk plan balances events across chunks) and on
    whole warps of 32 chunks when there are enough of them."""
    if n_chunks < world:
        raise ValueError(f"{n_chunks} chunks cannot be split over {world} ranks")
    unit = 32 if n_chunks >= 32 * world and n_chunks % 32 == 0 else 1
    n_units = n_chunks // unit
    cuts = [unit * ((n_units * r) // world) for r in range(world)] + [n_chunks]
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_spans(elem, group=None):
    """All-gather every rank's span element ([rows, NC] tensor, on the
    rank's GPU under NCCL or on the CPU under gloo) into [world, rows, NC]
    in rank (time) order."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    elem = elem.contiguous()
    parts = [torch.empty_like(elem) for _ in range(world)]
    dist.all_gather(parts, elem, group=group)
    return torch.stack(parts)


def time_sharded_loglik(model, theta, per_series=True, group=None, stream=None):
    """Log-likelihood of a one-series ``model`` split in time across the
    ranks of ``group``: this rank's chunk range, one all-gather, the fold.
    Every rank returns the same values (float64 CUDA tensor [rows])."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    c0, c1 = span_chunk_ranges(model.info["n_chunks"], world)[rank]
    elem = model.span_element(theta, c0, c1, per_series=per_series, stream=stream)
    return model.span_loglik(gather_spans(elem, group), stream=stream)
