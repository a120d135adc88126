"""Splitting one population over several GPUs, one process per GPU.

Cells are independent, so the closure, the learned closure, the adjoint and
the velocity update shard by cell with no collective on the data path: rank r
of W takes a contiguous range of cells holding about 1/W of the particles
(boundaries rounded to multiples of 32 cells, the tiles of the stored
factors), with its contiguous particle slice and offsets rebased to it.  The
velocity update's Philox counters continue across the slices when each rank
passes its slice's first global particle index as
fp_params.particle_offset, so the sharded run draws the variates of the
unsharded one.
"""

from __future__ import annotations

import numpy as np


def shard_bounds(offsets, world: int, rank: int, align: int = 32):
    """(c0, c1, p0, p1): the cells [c0, c1) and particles [p0, p1) of `rank`.
    The cut before rank r is the first cell whose offset reaches r/W of the
    particles, rounded down to a multiple of `align` (the last cut is the end),
    so the ranges are contiguous, ordered and cover every cell once."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    offsets = np.asarray(offsets, dtype=np.int64)
    n_cells = offsets.size - 1
    n_p = int(offsets[-1])

    def cut(r):
        if r <= 0:
            return 0
        if r >= world:
            return n_cells
        c = int(np.searchsorted(offsets, (n_p * r) // world, side="left"))
        return min(n_cells, (c // align) * align)

    c0, c1 = cut(rank), cut(rank + 1)
    return c0, c1, int(offsets[c0]), int(offsets[c1])


def shard_arrays(v, offsets, tau, world: int, rank: int, align: int = 32):
    """The rank's slice of a population held as arrays: velocities [3, p1-p0]
    (a copy, contiguous), offsets rebased to the slice, tau, and the slice's
    first global particle index (the Philox counter offset)."""
    c0, c1, p0, p1 = shard_bounds(offsets, world, rank, align)
    offsets = np.asarray(offsets, dtype=np.int64)
    return (np.ascontiguousarray(v[:, p0:p1]), offsets[c0:c1 + 1] - p0, np.asarray(tau)[c0:c1], p0,
            (c0, c1))
