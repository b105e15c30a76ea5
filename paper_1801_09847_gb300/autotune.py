"""Autotuner for batched registration: picks the grid cell size and the iteration kernel's launch form.

Two knobs, both free to choose because neither changes any result (the
correspondence search is exact for every cell size, and both launch forms run
the same arithmetic in the same order):

* cell size of the target grids, as a multiple of max_correspondence_distance;
* the launch form of the iteration kernel for the batch's size class
  (``o3g.TILE_LATENCY``: large shared-memory stage, 5 blocks per SM;
  ``o3g.TILE_THROUGHPUT``: smaller stage, 7 blocks per SM), pinned with
  ``o3g.set_tile_config``.

Block size (128 threads) and points per thread (1) are not searched: the tile
partition fixes the summation order of the block partials, so changing it
would change results in the last bits, which the two knobs above never do.

``tune_batch`` times a short batched call (a few iterations, CUDA events on
the current stream) for every candidate, pins the fastest form for the batch's
size class and returns the choice with all timings.  Grids built during tuning
are freed.
"""
from __future__ import annotations

import numpy as np

from . import o3g

DEFAULT_CELL_FACTORS = (0.75, 1.002, 1.5)
DEFAULT_FORMS = (o3g.TILE_LATENCY, o3g.TILE_THROUGHPUT)


def batch_tiles(srcs) -> int:
    """Work tiles (128 source points of one pair) of one batched launch."""
    return int(sum((int(s.shape[0]) + 127) // 128 for s in srcs))


def _build(tgts, nrms, cell):
    grids = []
    for t, n in zip(tgts, nrms):
        g = o3g.build_grid(t, cell)
        g.set_normals(n)
        grids.append(g)
    return grids


def tune_batch(tgts, nrms, srcs, max_corr_dist: float, iters: int = 5, reps: int = 2,
               cell_factors=DEFAULT_CELL_FACTORS, forms=DEFAULT_FORMS) -> dict:
    """Times o3g.icp_point_to_plane_batch for every (cell factor, launch form) on these pairs (device tensors:
    target points, target normals, sources) and pins the fastest form for the batch's size class.

    Returns dict(cell_factor, form, size_class, tiles, timings_ms={(cell_factor, form): ms per call}).
    """
    import torch
    cls = o3g.size_class(batch_tiles(srcs))
    previous = o3g.get_tile_config(cls)
    init = [np.eye(4)] * len(srcs)
    stream = torch.cuda.current_stream()
    timings = {}
    try:
        for cf in cell_factors:
            grids = _build(tgts, nrms, max_corr_dist * cf)
            try:
                for form in forms:
                    o3g.set_tile_config(cls, form)
                    o3g.icp_point_to_plane_batch(grids, srcs, init, max_corr_dist, iters)  # warm-up
                    best = float("inf")
                    for _ in range(reps):
                        e0 = torch.cuda.Event(enable_timing=True)
                        e1 = torch.cuda.Event(enable_timing=True)
                        e0.record(stream)
                        o3g.icp_point_to_plane_batch(grids, srcs, init, max_corr_dist, iters)
                        e1.record(stream)
                        e1.synchronize()
                        best = min(best, e0.elapsed_time(e1))
                    timings[(cf, form)] = best
            finally:
                for g in grids:
                    g.free()
    except Exception:
        o3g.set_tile_config(cls, previous)
        raise
    (cf, form), _ = min(timings.items(), key=lambda kv: kv[1])
    o3g.set_tile_config(cls, form)
    return dict(cell_factor=cf, form=form, size_class=cls, tiles=batch_tiles(srcs), timings_ms=timings)
