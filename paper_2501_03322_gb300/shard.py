"""Splitting one workload across GPUs (one process per GPU).

Source positions are independent (the paper's multi-GPU scaling, Sec. 4.4,
needs no communication between devices), so one flattened work list is cut
into contiguous ranges, one per rank, each rank integrates its range on its
own GPU, and the results are gathered.  The ranges are balanced by predicted
cost: the limb samples each position needed in a previous run (the method's
own work measure), or equal counts when there is none.  A contiguous cut
keeps every rank's inputs and outputs one slice of the caller's arrays.

The gather is a ``torch.distributed`` all-gather of the per-rank slices (NCCL
between GPUs, gloo on CPU), padded to the longest range.
"""
from __future__ import annotations

import numpy as np


def balanced_bounds(costs, nranks: int) -> np.ndarray:
    """Bounds b[0..nranks] (b[0] = 0, b[-1] = n) of contiguous ranges whose
    summed costs are as equal as a cut between positions allows: range r ends
    at the first position where the running cost reaches (r + 1)/nranks of
    the total.  `costs` is an int or a 1-D array (an int n means equal costs)."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    if np.isscalar(costs):
        n = int(costs)
        return np.array([(n * r) // nranks for r in range(nranks + 1)], dtype=np.int64)
    c = np.asarray(costs, dtype=np.float64)
    if c.ndim != 1 or (c < 0).any() or not np.isfinite(c).all():
        raise ValueError("costs must be a 1-D array of finite non-negative values")
    n = c.size
    total = c.sum()
    if total <= 0:
        return balanced_bounds(n, nranks)
    run = np.cumsum(c)
    b = np.zeros(nranks + 1, dtype=np.int64)
    for r in range(1, nranks):
        b[r] = int(np.searchsorted(run, total * r / nranks, side="left")) + 1
    b[nranks] = n
    return np.maximum.accumulate(np.minimum(b, n))


def gather(local, bounds, dist, device=None):
    """All-gather the per-rank result slices into the full array (every rank
    receives it).  `local` is this rank's slice (a 1-D torch tensor),
    `bounds` the common range bounds, `dist` torch.distributed."""
    import torch

    nranks = len(bounds) - 1
    sizes = np.diff(bounds)
    m = int(sizes.max()) if nranks else 0
    dev = device if device is not None else local.device
    pad = torch.zeros(m, dtype=local.dtype, device=dev)
    pad[: local.numel()] = local.to(dev)
    parts = [torch.empty_like(pad) for _ in range(nranks)]
    dist.all_gather(parts, pad)
    return torch.cat([p[: int(s)] for p, s in zip(parts, sizes)])


def run_sharded(n: int, compute, dist, costs=None, device=None):
    """Evaluate positions 0..n-1 split across the ranks of `dist`:
    compute(lo, hi) returns this rank's results for positions [lo, hi) as a
    1-D torch tensor; returns (the full gathered result, the bounds)."""
    rank, world = dist.get_rank(), dist.get_world_size()
    bounds = balanced_bounds(n if costs is None else costs, world)
    lo, hi = int(bounds[rank]), int(bounds[rank + 1])
    local = compute(lo, hi)
    if local.numel() != hi - lo:
        raise ValueError("compute(lo, hi) must return hi - lo values")
    return gather(local, bounds, dist, device), bounds
