"""Partition of the propagation workloads over GPUs, one process per GPU.

Particles are independent (paper Sec. 3.1: the module sequence of one particle never reads
another's state), so nothing is exchanged while they propagate:

* the batching form's field realisations are split by grid id: rank r builds and holds only
  the realisations in its block, and propagates only the particles that belong to them (their
  grid ids renumbered to the rank's own field list);
* other batches are split into contiguous blocks of particles;
* the one collective of the path is the differentiation form's gradient with respect to the
  field grid: every rank scatters its particles' share into its own copy, and one sum
  all-reduce gives every rank the whole gradient.

Host logic only: which rank owns what, and the reduction call.
"""
from __future__ import annotations

import numpy as np


def block_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[lo, hi) of rank's contiguous block when n items are split over `world` ranks (the
    first n % world ranks take one more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    q, r = divmod(int(n), int(world))
    lo = rank * q + min(rank, r)
    return lo, lo + q + (1 if rank < r else 0)


def grid_shard(n_grids: int, rank: int, world: int) -> np.ndarray:
    """Global ids of the field realisations held by `rank`."""
    lo, hi = block_range(n_grids, rank, world)
    return np.arange(lo, hi, dtype=np.int32)


def take_grid_shard(parts, grid_ids: np.ndarray):
    """The particles whose grid id is in `grid_ids`, with grid ids renumbered to positions in
    `grid_ids` (the rank's own field list); uids stay global."""
    grid_ids = np.asarray(grid_ids, dtype=np.int32)
    sel = np.isin(parts.grid_id, grid_ids)
    sub = parts.take(np.nonzero(sel)[0])
    local = np.full(int(grid_ids.max()) + 1 if grid_ids.size else 0, -1, dtype=np.int32)
    local[grid_ids] = np.arange(grid_ids.size, dtype=np.int32)
    sub.grid_id[:] = local[sub.grid_id]
    return sub


def allreduce_sum_(t, dist) -> None:
    """In-place sum over all ranks (the grid gradient of the differentiation form)."""
    if dist is not None and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
