"""Host side of the slab-sharded sweep (one tensor split along its first mode
across processes, one GPU each; the library's ifctn_sweep_exchange).

The library runs every kernel; this module only cuts a problem into slabs,
reassembles the factors, and provides an allreduce over torch.distributed
that gives the same bits on every process (an all-gather summed in process
order), as ifctn_sweep_exchange requires.
"""
from __future__ import annotations

import numpy as np

from . import inputs as inp


def slab_bounds(I0: int, world: int, rank: int):
    """Rows [lo, hi) of the first mode held by `rank` (contiguous, sizes
    differing by at most one)."""
    lo = I0 * rank // world
    hi = I0 * (rank + 1) // world
    return lo, hi


def slab_factors(G, dims, R, lo, hi):
    """The slab problem's packed factors: the columns lo..hi-1 of every
    G_{0,l}, the other factors whole."""
    N = len(dims)
    sdims = (hi - lo,) + tuple(dims[1:])
    F = inp.unpack_factors(np.asarray(G, dtype=np.float64), dims, R)
    out = np.empty(inp.factor_size(sdims, R), dtype=np.float64)
    S = inp.unpack_factors(out, sdims, R)
    for k in range(N):
        for l in range(N):
            if l != k:
                S[(k, l)][...] = F[(k, l)][:, lo:hi] if k == 0 else F[(k, l)]
    return out


def merge_factors(slabs, dims, R, bounds):
    """Whole-problem factors from the slabs' factors: G_{0,l} columns from
    their slabs, every other factor from slab 0 (the slabs agree on them)."""
    N = len(dims)
    out = np.empty(inp.factor_size(dims, R), dtype=np.float64)
    F = inp.unpack_factors(out, dims, R)
    for (lo, hi), G in zip(bounds, slabs):
        S = inp.unpack_factors(np.asarray(G), (hi - lo,) + tuple(dims[1:]), R)
        for k in range(N):
            for l in range(N):
                if l == k:
                    continue
                if k == 0:
                    F[(k, l)][:, lo:hi] = S[(k, l)]
                elif (lo, hi) == bounds[0]:
                    F[(k, l)][...] = S[(k, l)]
    return out


def ordered_allreduce(dist, group=None):
    """An allreduce for ifctn_sweep_exchange over torch.distributed: every
    process all-gathers the values and sums them in process order, so every
    process holds the same bits (a library collective may sum in another
    order on each process)."""
    import torch

    def allreduce(values):
        t = torch.from_numpy(np.array(values, dtype=np.float64, copy=True))
        world = dist.get_world_size(group)
        parts = [torch.empty_like(t) for _ in range(world)]
        dist.all_gather(parts, t, group=group)
        acc = parts[0].clone()
        for p in parts[1:]:
            acc += p
        values[...] = acc.numpy()

    return allreduce
