"""Autotuner for batched registration: grid cell size, launch form and points per thread.

Three knobs:

* cell size of the target grids, as a multiple of max_correspondence_distance;
* the launch form of the iteration kernel for the batch's size class of work
  tiles (``o3g.TILE_LATENCY``: large shared-memory stage, 5 blocks per SM;
  ``o3g.TILE_THROUGHPUT``: per-thread searches from global memory, 9 blocks
  per SM, candidate lists),
  pinned with ``o3g.set_tile_config``;
* points per thread (1, 2 or 4: a tile of the iteration kernel is that many
  groups of 128 spatially sorted source points) for each size class of the
  PAIRS in the batch (floor(log2(source points))), pinned with
  ``o3g.set_points_per_thread``.

The first two never change a result (the correspondence search is exact for
every cell size, and both launch forms run the same arithmetic in the same
order).  Points per thread sets how a pair's sums are grouped into block
partials, so it changes results in the last bits; it is a property of the
pair's size class, so a pair tiles the same way alone, in a batch and in the
server.  Threads per block stay 128: the shared-memory stage, the transposed
reduction of the rows and the solve are laid out for four warps, and larger
tiles come from points per thread.

``tune_batch`` times a short batched call (a few iterations, CUDA events on
the current stream): every (cell factor, launch form) with automatic points
per thread, then, from the best of those, each pair size class in turn (the
classes holding the most points first) with 1, 2 and 4 points per thread.  It
pins the choices and returns them with all timings.  Grids built during tuning
are freed.
"""
from __future__ import annotations

import numpy as np

from . import o3g

DEFAULT_CELL_FACTORS = (0.75, 1.002, 1.5)
DEFAULT_FORMS = (o3g.TILE_LATENCY, o3g.TILE_THROUGHPUT)
DEFAULT_PPTS = (1, 2, 4)


def batch_tiles(srcs) -> int:
    """Work tiles of one batched launch at one point per thread (128 source points of one pair each)."""
    return int(sum((int(s.shape[0]) + 127) // 128 for s in srcs))


def auto_ppt(n: int) -> int:
    """The library's automatic points per thread for a pair of n source points."""
    return 4 if n >= 1 << 20 else (2 if n >= 1 << 18 else 1)


def _build(tgts, nrms, cell):
    grids = []
    for t, n in zip(tgts, nrms):
        g = o3g.build_grid(t, cell)
        g.set_normals(n)
        grids.append(g)
    return grids


def _time(grids, srcs, init, max_corr_dist, iters, reps):
    import torch
    stream = torch.cuda.current_stream()
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
    return best


def tune_batch(tgts, nrms, srcs, max_corr_dist: float, iters: int = 5, reps: int = 2,
               cell_factors=DEFAULT_CELL_FACTORS, forms=DEFAULT_FORMS, ppts=DEFAULT_PPTS) -> dict:
    """Times o3g.icp_point_to_plane_batch on these pairs (device tensors: target points, target normals, sources)
    for every (cell factor, launch form), then points per thread per pair size class, and pins the fastest.

    Returns dict(cell_factor, form, size_class, tiles, ppt={pair size class: points per thread (0: automatic)},
    timings_ms={(cell_factor, form): ms per call}, ppt_timings_ms={(pair size class, ppt): ms per call}).
    """
    cls = o3g.size_class(batch_tiles(srcs))
    pair_classes = {}
    for s in srcs:
        c = o3g.pair_size_class(int(s.shape[0]))
        pair_classes[c] = pair_classes.get(c, 0) + int(s.shape[0])
    previous = o3g.get_tile_config(cls)
    previous_ppt = {c: o3g.get_points_per_thread(c) for c in pair_classes}
    init = [np.eye(4)] * len(srcs)
    timings, ppt_timings = {}, {}
    try:
        for c in pair_classes:
            o3g.set_points_per_thread(c, 0)
        for cf in cell_factors:
            grids = _build(tgts, nrms, max_corr_dist * cf)
            try:
                for form in forms:
                    o3g.set_tile_config(cls, form)
                    timings[(cf, form)] = _time(grids, srcs, init, max_corr_dist, iters, reps)
            finally:
                for g in grids:
                    g.free()
        (cf, form), best = min(timings.items(), key=lambda kv: kv[1])
        o3g.set_tile_config(cls, form)
        chosen = {}
        grids = _build(tgts, nrms, max_corr_dist * cf)
        try:
            for c in sorted(pair_classes, key=lambda k: -pair_classes[k]):
                best_ppt, best_ms = 0, best
                for ppt in ppts:
                    o3g.set_points_per_thread(c, ppt)
                    ms = _time(grids, srcs, init, max_corr_dist, iters, reps)
                    ppt_timings[(c, ppt)] = ms
                    if ms < best_ms:
                        best_ppt, best_ms = ppt, ms
                o3g.set_points_per_thread(c, best_ppt)
                chosen[c] = best_ppt
                best = best_ms
        finally:
            for g in grids:
                g.free()
        # the launches then have this many tiles: pin the chosen form for their size class too
        tiles = 0
        for s in srcs:
            n = int(s.shape[0])
            ppt = chosen.get(o3g.pair_size_class(n)) or auto_ppt(n)
            tiles += max(1, -(-n // (128 * ppt)))
        o3g.set_tile_config(o3g.size_class(tiles), form)
    except Exception:
        o3g.set_tile_config(cls, previous)
        for c, v in previous_ppt.items():
            o3g.set_points_per_thread(c, v)
        raise
    return dict(cell_factor=cf, form=form, size_class=cls, tiles=batch_tiles(srcs), ppt=chosen,
                timings_ms=timings, ppt_timings_ms=ppt_timings)
