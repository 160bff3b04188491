"""Multi-GPU layout: signals are independent, so a batch is split across ranks with no exchange on
the data path.  Each rank plans and recovers only its own signals; results come back to the host
and are gathered once at the end (torch.distributed object gather, any backend).

The split is longest-processing-time first: signals sorted by estimated work (samples per
iteration times an iteration estimate), each assigned to the rank with the least work so far.
"""
from __future__ import annotations

import math

import numpy as np


def estimated_work(dims, T=None):
    """Per-signal work estimate: (D+1) L samples per iteration times min(T, 8) iterations."""
    dims = np.asarray(dims, np.int64)
    out = np.zeros(dims.shape[0], np.float64)
    for b, d in enumerate(dims):
        L = math.lcm(*[int(v) for v in d])
        t = 8 if T is None else min(int(T[b]), 8)
        out[b] = (len(d) + 1) * L * t
    return out


def lpt_partition(work, world):
    """Assign item indices to `world` bins, longest first to the currently lightest bin.
    Returns a list of sorted index arrays (one per rank); deterministic (ties by index)."""
    work = np.asarray(work, np.float64)
    order = sorted(range(len(work)), key=lambda i: (-work[i], i))
    load = [0.0] * world
    parts = [[] for _ in range(world)]
    for i in order:
        r = min(range(world), key=lambda q: (load[q], q))
        parts[r].append(i)
        load[r] += work[i]
    return [np.asarray(sorted(p), np.int64) for p in parts]


def shard(dims, world, rank, T=None):
    """Indices of the signals rank `rank` of `world` processes."""
    return lpt_partition(estimated_work(dims, T), world)[rank]


def gather_results(results, indices, world, rank, group=None):
    """Gather {signal index: result} from every rank to rank 0 (host objects).  Returns the merged
    dict on rank 0 and None elsewhere."""
    import torch.distributed as dist
    local = {int(i): r for i, r in zip(indices, results)}
    if world == 1:
        return local
    buf = [None] * world if rank == 0 else None
    dist.gather_object(local, buf, dst=0, group=group)
    if rank != 0:
        return None
    merged = {}
    for part in buf:
        merged.update(part)
    return merged
