"""Thin ctypes binding of libo3g.so (C ABI in include/o3g.h).

Argument marshalling only: every step of the registration path runs in the
library's CUDA kernels.  PyTorch provides device memory and the current
stream.  There is no CPU fallback: if libo3g.so is missing or cannot be loaded,
every call raises.

Names follow the C ABI and the paper's API (Sec. 3.3 of arXiv 1801.09847):
``build_grid`` (the kd-tree's replacement), ``estimate_normals``,
``knn_hybrid``, ``correspondences``, ``normal_equations``,
``icp_point_to_plane_grid``, ``icp_point_to_plane`` and
``register_point_to_plane_host``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libo3g.so")

OK, WARN_DEGENERATE, WARN_FEW_CORR = 0, 1, 2
ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NONFINITE, ERR_TIMEOUT = -1, -2, -3, -4, -5
MAX_NN = 64
STATUS_NAMES = {0: "OK", 1: "WARN_DEGENERATE", 2: "WARN_FEW_CORR", -1: "ERR_ARG", -2: "ERR_OOM",
                -3: "ERR_CUDA", -4: "ERR_NONFINITE", -5: "ERR_TIMEOUT"}


class O3GError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None
_lock = threading.Lock()
_vp, _i64, _i32, _f32, _f64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_double
_f64p = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)

_SIGNATURES = {
    "o3g_last_error": ([], ctypes.c_char_p),
    "o3g_abi_version": ([], _i32),
    "o3g_build_grid": ([_vp, _i64, _i32, _f32, _vp, ctypes.POINTER(_vp)], _i32),
    "o3g_free_grid": ([_vp], _i32),
    "o3g_grid_info": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_f32)], _i32),
    "o3g_grid_set_normals": ([_vp, _vp, _i64, _i32, _vp], _i32),
    "o3g_knn_hybrid": ([_vp, _vp, _i64, _i32, _f32, _i32, _vp, _vp, _vp, _vp], _i32),
    "o3g_estimate_normals": ([_vp, _f32, _i32, _vp, _vp, _i32, _vp], _i32),
    "o3g_correspondences": ([_vp, _vp, _i64, _i32, _f64p, _f32, _vp, _vp, _vp], _i32),
    "o3g_normal_equations": ([_vp, _vp, _i64, _i32, _f64p, _f32, _f64p, _f64p, _f64p, _vp], _i32),
    "o3g_normal_equations_ex": ([_vp, _vp, _i64, _i32, _f64p, _f32, _i32, _f64p, _f64p, _f64p, _vp], _i32),
    "o3g_estimate_normals_batch": ([_i32, _vp, _vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "o3g_knn_hybrid_batch": ([_i32, _vp, _vp, _vp, _vp, _vp, _i32, _vp, _vp, _vp, _vp], _i32),
    "o3g_set_tile_config": ([_i32, _i32], _i32),
    "o3g_get_tile_config": ([_i32], _i32),
    "o3g_set_points_per_thread": ([_i32, _i32], _i32),
    "o3g_get_points_per_thread": ([_i32], _i32),
    "o3g_evaluate_poses": ([_vp, _vp, _i64, _i32, _i32, _f64p, _f64, _f64p, _f64p,
                            ctypes.POINTER(ctypes.c_int64), _vp], _i32),
    "o3g_voxel_down_sample": ([_vp, _i64, _i32, _f32, _vp, _vp, ctypes.POINTER(ctypes.c_int64), _vp], _i32),
    "o3g_icp_point_to_point_grid": ([_vp, _vp, _i64, _i32, _f64p, _f64, _i32, _f64, _f64p, _f64p, _f64p, _i32p, _vp],
                                    _i32),
    "o3g_icp_point_to_plane_grid_ex": ([_vp, _vp, _i64, _i32, _f64p, _f64, _i32, _f64, _i32, _f64p, _f64p, _f64p,
                                        _i32p, _vp], _i32),
    "o3g_icp_point_to_plane_grid": ([_vp, _vp, _i64, _i32, _f64p, _f64, _i32, _f64, _f64p, _f64p, _f64p, _i32p, _vp],
                                    _i32),
    "o3g_icp_point_to_plane_grid_corr": ([_vp, _vp, _i64, _i32, _f64p, _f64, _i32, _f64, _i32, _f64p, _f64p, _f64p,
                                          _i32p, _vp, _vp, _vp], _i32),
    "o3g_icp_point_to_plane": ([_vp, _i64, _i32, _vp, _i64, _i32, _vp, _i64, _i32, _f64p, _f64, _i32, _f64p, _f64p,
                                _f64p], _i32),
    "o3g_register_point_to_plane": ([_vp, _i64, _i32, _vp, _i64, _i32, _vp, _i32, _f32, _i32, _f64p, _f64, _i32, _f64,
                                     _f64p, _f64p, _f64p, ctypes.POINTER(_i32), _vp], _i32),
    "o3g_register_point_to_plane_host": ([_vp, _i64, _vp, _i64, _vp, _f32, _i32, _f64p, _f64, _i32, _f64, _f64p,
                                          _f64p, _f64p, _i32p, _vp], _i32),
    "o3g_icp_point_to_plane_batch": ([_i32, _vp, _vp, _vp, _vp, _f64p, _f64p, _i32, _f64, _f64p, _f64p, _f64p, _i32p,
                                      _i32p, _vp], _i32),
    "o3g_server_create": ([_i32, _i64, _vp, ctypes.POINTER(_vp)], _i32),
    "o3g_server_request_bytes": ([_i64, _i64], _i64),
    "o3g_server_destroy": ([_vp], _i32),
    "o3g_server_submit": ([_vp, _vp, _i64, _vp, _i64, _vp, _f32, _i32, _f64p, _f64, _i32, _f64,
                           ctypes.POINTER(_i64)], _i32),
    "o3g_server_step": ([_vp, _i32p, _i32p, _i32p], _i32),
    "o3g_server_poll": ([_vp, _i64, _i32p, _f64p, _f64p, _f64p, _i32p, _i32p], _i32),
    "o3g_server_completed": ([_vp, _vp, _i32, _i32p], _i32),
    "o3g_icp_point_to_plane_grid_noalloc": ([_vp, _vp, _i64, _i32, _f64p, _f64, _i32, _f64, _f64p, _f64p, _f64p,
                                             _i32p, _vp], _i32),
    "o3g_launch_count": ([], _i64),
    "o3g_timing_enable": ([_i32], _i32),
    "o3g_timing_read": ([_i32, _f64p, ctypes.POINTER(_i64), _i32], _i32),
}

KERNEL_ICP_CORR, KERNEL_ICP_SOLVE, KERNEL_NORMALS, KERNEL_GRID, KERNEL_ICP_BATCH, KERNEL_VOXEL, KERNEL_EVAL = range(7)
# o3g_precision
PREC_F32_COMPENSATED, PREC_F64 = 0, 1
_PRECISIONS = {"f32": PREC_F32_COMPENSATED, "f64": PREC_F64}


def _precision(precision) -> int:
    if precision in _PRECISIONS:
        return _PRECISIONS[precision]
    if precision in (PREC_F32_COMPENSATED, PREC_F64):
        return int(precision)
    raise ValueError(f"unknown precision {precision!r} (use 'f32' or 'f64')")


def launch_count() -> int:
    """Kernels libo3g.so has launched since it was loaded."""
    return int(lib().o3g_launch_count())


def timing_enable(on: bool = True) -> None:
    """Bracket each launch of the timed kernels with CUDA events on their launching stream."""
    lib().o3g_timing_enable(1 if on else 0)


def timing_read(kind: int, reset: bool = True) -> tuple[float, int]:
    """(summed device milliseconds, launches) recorded for one kernel kind since the last reset."""
    ms, n = _f64(), _i64()
    _check(lib().o3g_timing_read(int(kind), ctypes.byref(ms), ctypes.byref(n), 1 if reset else 0),
           "o3g_timing_read")
    return ms.value, n.value


def lib():
    """Loads libo3g.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libo3g.so not built ({LIB_PATH}); run __graft_entry__.build()")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in _SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def last_error() -> str:
    return lib().o3g_last_error().decode(errors="replace")


def _check(st: int, where: str) -> int:
    if st < 0:
        raise O3GError(st, where, last_error())
    return st


def _torch():
    import torch
    return torch


def _stream(stream) -> ctypes.c_void_p:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _cloud(t, name: str):
    """(device pointer, n, stride) of an N x k (k >= 3) float32 CUDA tensor with unit inner stride."""
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.float32:
        raise TypeError(f"{name} must be a float32 CUDA tensor")
    if t.dim() != 2 or t.shape[1] < 3 or (t.shape[0] > 1 and t.stride(1) != 1):
        raise ValueError(f"{name} must be N x k (k >= 3) with contiguous rows")
    stride = t.stride(0) if t.shape[0] > 1 else max(3, t.shape[1])
    return ctypes.c_void_p(t.data_ptr() if t.numel() else 0), t.shape[0], stride


def _pose(T) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(T, dtype=np.float64).reshape(16))


def _pp(a: np.ndarray):
    return a.ctypes.data_as(_f64p)


class Grid:
    """Device uniform grid over one cloud (o3g_build_grid); freed with the object."""

    def __init__(self, handle: int, n: int, stream):
        self._h = ctypes.c_void_p(handle)
        self.n = n
        self._stream = stream

    @property
    def handle(self) -> ctypes.c_void_p:
        if not self._h:
            raise RuntimeError("grid already freed")
        return self._h

    def info(self):
        n, cell = _i64(), _f32()
        _check(lib().o3g_grid_info(self.handle, ctypes.byref(n), ctypes.byref(cell)), "o3g_grid_info")
        return n.value, cell.value

    def free(self):
        if self._h:
            lib().o3g_free_grid(self._h)
            self._h = ctypes.c_void_p(0)

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def set_normals(self, nrm, stream=None):
        p, n, stride = _cloud(nrm, "normals")
        _check(lib().o3g_grid_set_normals(self.handle, p, n, stride, _stream(stream)), "o3g_grid_set_normals")

    def estimate_normals(self, radius: float, max_nn: int, viewpoint=(0.0, 0.0, 0.0), out=None, stream=None):
        """estimate_normals(pc, KDTreeSearchParamHybrid(radius, max_nn)); returns N x 3 normals (input order).

        out=None allocates the result; out=False keeps the normals in the grid only and returns None.
        """
        torch = _torch()
        if out is False:
            p, stride = _vp(0), 3
        else:
            if out is None:
                out = torch.empty((self.n, 3), dtype=torch.float32, device="cuda")
            p, n, stride = _cloud(out, "out")
            if n != self.n:
                raise ValueError("out must have one row per grid point")
        vp = (ctypes.c_float * 3)(*[float(v) for v in viewpoint])
        _check(lib().o3g_estimate_normals(self.handle, float(radius), int(max_nn), ctypes.cast(vp, _vp), p, stride,
                                          _stream(stream)), "o3g_estimate_normals")
        return None if out is False else out


def build_grid(xyz, cell_size: float, stream=None) -> Grid:
    p, n, stride = _cloud(xyz, "xyz")
    h = ctypes.c_void_p()
    _check(lib().o3g_build_grid(p, n, stride, float(cell_size), _stream(stream), ctypes.byref(h)), "o3g_build_grid")
    return Grid(h.value, n, stream)


def knn_hybrid(grid: Grid, queries, radius: float, max_nn: int, stream=None):
    """KDTreeSearchParamHybrid(radius, max_nn) search: (idx int32 [nq, max_nn], d2 [nq, max_nn], count [nq])."""
    torch = _torch()
    p, nq, stride = _cloud(queries, "queries")
    idx = torch.empty((nq, max_nn), dtype=torch.int32, device="cuda")
    d2 = torch.empty((nq, max_nn), dtype=torch.float32, device="cuda")
    cnt = torch.empty((nq,), dtype=torch.int32, device="cuda")
    _check(lib().o3g_knn_hybrid(grid.handle, p, nq, stride, float(radius), int(max_nn), _vp(idx.data_ptr()),
                                _vp(d2.data_ptr()), _vp(cnt.data_ptr()), _stream(stream)), "o3g_knn_hybrid")
    return idx, d2, cnt


def correspondences(grid: Grid, src, T, max_corr_dist: float, stream=None):
    """Transform + fixed-radius NN at pose T: (corr int32 [ns], d2 float32 [ns])."""
    torch = _torch()
    p, ns, stride = _cloud(src, "src")
    corr = torch.empty((ns,), dtype=torch.int32, device="cuda")
    d2 = torch.empty((ns,), dtype=torch.float32, device="cuda")
    Tp = _pose(T)
    _check(lib().o3g_correspondences(grid.handle, p, ns, stride, _pp(Tp), float(max_corr_dist), _vp(corr.data_ptr()),
                                     _vp(d2.data_ptr()), _stream(stream)), "o3g_correspondences")
    return corr, d2


def normal_equations(grid: Grid, src, T, max_corr_dist: float, stream=None, precision="f32"):
    """J^T J (6x6), J^T r (6), (sum r^2, sum d2, |C|) at pose T (Eq. 2).

    precision "f32" (float32 terms, compensated block sums) or "f64" (all float64).
    """
    p, ns, stride = _cloud(src, "src")
    A = np.zeros(36)
    b = np.zeros(6)
    stats = np.zeros(3)
    Tp = _pose(T)
    _check(lib().o3g_normal_equations_ex(grid.handle, p, ns, stride, _pp(Tp), float(max_corr_dist),
                                         _precision(precision), _pp(A), _pp(b), _pp(stats), _stream(stream)),
           "o3g_normal_equations_ex")
    return A.reshape(6, 6), b, stats


def _result(st, T, fit, rmse, iters):
    return dict(status=st, T=T.reshape(4, 4), fitness=fit.value, rmse=rmse.value,
                iters=iters.value if iters is not None else None)


def icp_point_to_plane_grid(grid: Grid, src, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                            stream=None, precision="f32", correspondences: bool = False) -> dict:
    """registration_icp(..., TransformationEstimationPointToPlane()) against a resident target grid.

    precision "f32" (float32 terms, compensated block sums) or "f64" (all float64).  correspondences=True adds the
    correspondence set at the final pose: "corr" (int32 [ns], original target index or -1) and "d2" (float32 [ns])
    as CUDA tensors (o3g_icp_point_to_plane_grid_corr).
    """
    p, ns, stride = _cloud(src, "src")
    T0 = _pose(init_T)
    T = np.zeros(16)
    fit, rmse, iters = _f64(), _f64(), _i32()
    if correspondences:
        torch = _torch()
        corr = torch.empty((ns,), dtype=torch.int32, device="cuda")
        d2 = torch.empty((ns,), dtype=torch.float32, device="cuda")
        st = lib().o3g_icp_point_to_plane_grid_corr(grid.handle, p, ns, stride, _pp(T0), float(max_corr_dist),
                                                    int(max_iter), float(eps), _precision(precision), _pp(T),
                                                    ctypes.byref(fit), ctypes.byref(rmse), ctypes.byref(iters),
                                                    _vp(corr.data_ptr()), _vp(d2.data_ptr()), _stream(stream))
        st = _check(st, "o3g_icp_point_to_plane_grid_corr")
        out = _result(st, T, fit, rmse, iters)
        out["corr"], out["d2"] = corr, d2
        return out
    if _precision(precision) == PREC_F32_COMPENSATED:
        st = lib().o3g_icp_point_to_plane_grid(grid.handle, p, ns, stride, _pp(T0), float(max_corr_dist),
                                               int(max_iter), float(eps), _pp(T), ctypes.byref(fit),
                                               ctypes.byref(rmse), ctypes.byref(iters), _stream(stream))
    else:
        st = lib().o3g_icp_point_to_plane_grid_ex(grid.handle, p, ns, stride, _pp(T0), float(max_corr_dist),
                                                  int(max_iter), float(eps), PREC_F64, _pp(T), ctypes.byref(fit),
                                                  ctypes.byref(rmse), ctypes.byref(iters), _stream(stream))
    st = _check(st, "o3g_icp_point_to_plane_grid")
    return _result(st, T, fit, rmse, iters)


def _ptrs(values):
    arr = (ctypes.c_void_p * max(len(values), 1))()
    for k, v in enumerate(values):
        arr[k] = v
    return arr


def estimate_normals_batch(grids, radius, max_nn: int, viewpoints=None, outs=None, stream=None) -> None:
    """Normals of many clouds in one launch (o3g_estimate_normals_batch); each grid then carries its normals.

    radius: one per grid or a scalar; viewpoints: n x 3 or None (origins); outs: optional list of float32 CUDA
    tensors (n_c x k, k >= 3, or None entries) that also receive the normals by original index."""
    n = len(grids)
    rad = np.ascontiguousarray(np.broadcast_to(np.asarray(radius, np.float32), (n,)))
    vp = None if viewpoints is None else np.ascontiguousarray(np.asarray(viewpoints, np.float32).reshape(n, 3))
    handles = _ptrs([g.handle.value for g in grids])
    out_ptrs, strides = None, None
    if outs is not None:
        vals, st = [], np.full(max(n, 1), 3, np.int32)
        for k, o in enumerate(outs):
            if o is None:
                vals.append(None)
                continue
            p, m, stride = _cloud(o, f"outs[{k}]")
            if m != grids[k].info()[0]:
                raise ValueError(f"outs[{k}] must have one row per point of grids[{k}]")
            vals.append(p.value)
            st[k] = stride
        out_ptrs, strides = _ptrs(vals), st
    _check(lib().o3g_estimate_normals_batch(n, handles, rad.ctypes.data_as(ctypes.c_void_p), int(max_nn),
                                            vp.ctypes.data_as(ctypes.c_void_p) if vp is not None else None,
                                            out_ptrs, strides.ctypes.data_as(ctypes.c_void_p) if strides is not None
                                            else None, _stream(stream)), "o3g_estimate_normals_batch")


def knn_hybrid_batch(grids, queries, radius, max_nn: int, stream=None) -> list:
    """Hybrid kNN of many query sets against their grids in one launch: [(idx, d2, cnt)] per set."""
    torch = _torch()
    n = len(grids)
    rad = np.ascontiguousarray(np.broadcast_to(np.asarray(radius, np.float32), (n,)))
    qp, nq, st, outs = [], np.zeros(max(n, 1), np.int64), np.zeros(max(n, 1), np.int32), []
    for k, q in enumerate(queries):
        p, m, stride = _cloud(q, f"queries[{k}]")
        qp.append(p.value)
        nq[k], st[k] = m, stride
        outs.append((torch.empty((m, max_nn), dtype=torch.int32, device="cuda"),
                     torch.empty((m, max_nn), dtype=torch.float32, device="cuda"),
                     torch.empty((m,), dtype=torch.int32, device="cuda")))
    _check(lib().o3g_knn_hybrid_batch(n, _ptrs([g.handle.value for g in grids]), _ptrs(qp),
                                      nq.ctypes.data_as(ctypes.c_void_p), st.ctypes.data_as(ctypes.c_void_p),
                                      rad.ctypes.data_as(ctypes.c_void_p), int(max_nn),
                                      _ptrs([o[0].data_ptr() for o in outs]), _ptrs([o[1].data_ptr() for o in outs]),
                                      _ptrs([o[2].data_ptr() for o in outs]), _stream(stream)),
           "o3g_knn_hybrid_batch")
    return outs


TILE_AUTO, TILE_LATENCY, TILE_THROUGHPUT = 0, 1, 2


def size_class(tiles: int) -> int:
    """floor(log2(tiles)) clamped to 0..31: the index o3g_set_tile_config uses."""
    return max(0, min(31, int(tiles).bit_length() - 1))


def set_tile_config(size_class: int, cfg: int) -> None:
    """Pins the iteration kernel's launch form for one size class (TILE_AUTO / TILE_LATENCY / TILE_THROUGHPUT)."""
    _check(lib().o3g_set_tile_config(int(size_class), int(cfg)), "o3g_set_tile_config")


def get_tile_config(size_class: int) -> int:
    return _check(lib().o3g_get_tile_config(int(size_class)), "o3g_get_tile_config")


def pair_size_class(n_points: int) -> int:
    """floor(log2(source points)) clamped to 0..31: the index o3g_set_points_per_thread uses."""
    return max(0, min(31, int(n_points).bit_length() - 1))


def set_points_per_thread(size_class: int, ppt: int) -> None:
    """Pins the points per thread (0 automatic, 1, 2 or 4) of the pairs of one size class (o3g_set_points_per_thread)."""
    _check(lib().o3g_set_points_per_thread(int(size_class), int(ppt)), "o3g_set_points_per_thread")


def get_points_per_thread(size_class: int) -> int:
    return _check(lib().o3g_get_points_per_thread(int(size_class)), "o3g_get_points_per_thread")


def evaluate_poses(grid: Grid, src, poses, max_corr_dist: float, stream=None):
    """Hypothesis validation (Sec. 3.3, RANSAC): fitness, inlier rmse and inlier count of the whole source at each
    4x4 pose.  Returns (fitness [H], rmse [H], inliers [H]) as numpy arrays."""
    p, ns, stride = _cloud(src, "src")
    P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
    H = len(P)
    fit = np.zeros(max(H, 1))
    rmse = np.zeros(max(H, 1))
    cnt = np.zeros(max(H, 1), np.int64)
    _check(lib().o3g_evaluate_poses(grid.handle, p, ns, stride, H, _pp(P if H else np.zeros((1, 16))),
                                    float(max_corr_dist), _pp(fit), _pp(rmse),
                                    cnt.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _stream(stream)),
           "o3g_evaluate_poses")
    return fit[:H], rmse[:H], cnt[:H]


def voxel_down_sample(pts, voxel: float, stream=None, with_counts: bool = False):
    """voxel_down_sample (Sec. 3.1, Fig. 1) on the GPU: centroids (float32 [M, 3], device) of the occupied voxels
    in increasing (ix, iy, iz) order, and with_counts=True also the points per voxel (int32 [M])."""
    torch = _torch()
    p, n, stride = _cloud(pts, "pts")
    out = torch.empty((max(n, 1), 3), dtype=torch.float32, device="cuda")
    cnt = torch.empty((max(n, 1),), dtype=torch.int32, device="cuda") if with_counts else None
    m = ctypes.c_int64()
    _check(lib().o3g_voxel_down_sample(p, n, stride, float(voxel), _vp(out.data_ptr()),
                                       _vp(cnt.data_ptr()) if cnt is not None else None, ctypes.byref(m),
                                       _stream(stream)), "o3g_voxel_down_sample")
    out = out[: m.value]
    return (out, cnt[: m.value]) if with_counts else out


def icp_point_to_point_grid(grid: Grid, src, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                            stream=None) -> dict:
    """registration_icp(..., TransformationEstimationPointToPoint()) against a resident target grid
    (normals not needed).  Returns dict(status, T, fitness, rmse, iters)."""
    p, ns, stride = _cloud(src, "src")
    T0 = _pose(init_T)
    T = np.zeros(16)
    fit, rmse, iters = _f64(), _f64(), _i32()
    st = _check(lib().o3g_icp_point_to_point_grid(grid.handle, p, ns, stride, _pp(T0), float(max_corr_dist),
                                                  int(max_iter), float(eps), _pp(T), ctypes.byref(fit),
                                                  ctypes.byref(rmse), ctypes.byref(iters), _stream(stream)),
                "o3g_icp_point_to_point_grid")
    return _result(st, T, fit, rmse, iters)


def icp_point_to_plane_batch(grids, srcs, init_Ts, max_corr_dists, max_iter: int, eps: float = 0.0,
                             stream=None) -> list:
    """Many independent registrations in one batched call (o3g_icp_point_to_plane_batch).

    grids: target Grids with normals; srcs: device source clouds; init_Ts: 4x4 poses;
    max_corr_dists: one radius per pair or a scalar.  Returns one result dict per pair.
    """
    n = len(grids)
    if len(srcs) != n or len(init_Ts) != n:
        raise ValueError("grids, srcs and init_Ts must have one entry per pair")
    radii = np.broadcast_to(np.asarray(max_corr_dists, np.float64), (n,)).copy()
    handles = (ctypes.c_void_p * max(n, 1))(*[g.handle.value for g in grids])
    ptrs = (ctypes.c_void_p * max(n, 1))()
    ns = np.zeros(max(n, 1), np.int64)
    strides = np.zeros(max(n, 1), np.int32)
    for k, src in enumerate(srcs):
        p, m, stride = _cloud(src, f"srcs[{k}]")
        ptrs[k] = p.value
        ns[k] = m
        strides[k] = stride
    T0 = np.ascontiguousarray(np.stack([np.asarray(T, np.float64).reshape(16) for T in init_Ts]) if n else
                              np.zeros((1, 16)))
    T = np.zeros((max(n, 1), 16))
    fit = np.zeros(max(n, 1))
    rmse = np.zeros(max(n, 1))
    iters = np.zeros(max(n, 1), np.int32)
    status = np.zeros(max(n, 1), np.int32)
    _check(lib().o3g_icp_point_to_plane_batch(n, ctypes.cast(handles, _vp), ctypes.cast(ptrs, _vp),
                                              ns.ctypes.data_as(_vp), strides.ctypes.data_as(_vp), _pp(T0),
                                              _pp(radii), int(max_iter), float(eps), _pp(T), _pp(fit), _pp(rmse),
                                              iters.ctypes.data_as(_i32p), status.ctypes.data_as(_i32p),
                                              _stream(stream)), "o3g_icp_point_to_plane_batch")
    return [dict(status=int(status[k]), T=T[k].reshape(4, 4), fitness=float(fit[k]), rmse=float(rmse[k]),
                 iters=int(iters[k])) for k in range(n)]


class Server:
    """Continuous-batching registration server (o3g_server_*): submit, step, poll."""

    @staticmethod
    def request_bytes(ns: int, nt: int) -> int:
        """Device-memory estimate a request of ns source / nt target points is admitted against."""
        v = int(lib().o3g_server_request_bytes(int(ns), int(nt)))
        if v < 0:
            raise O3GError(ERR_ARG, "o3g_server_request_bytes", "negative or oversized cloud size")
        return v

    def __init__(self, max_active: int = 64, hbm_budget_bytes: int = 8 << 30, stream=None):
        h = _vp()
        _check(lib().o3g_server_create(int(max_active), int(hbm_budget_bytes), _stream(stream), ctypes.byref(h)),
               "o3g_server_create")
        self._h = h

    def close(self):
        if self._h:
            lib().o3g_server_destroy(self._h)
            self._h = _vp(0)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _host(a, name):
        if a is None:
            return None, 0
        arr = np.ascontiguousarray(a, dtype=np.float32)
        if arr.size and (arr.ndim != 2 or arr.shape[1] != 3):
            raise ValueError(f"{name} must be N x 3")
        return arr, (arr.shape[0] if arr.size else 0)

    def submit(self, src, tgt, tgt_nrm=None, init_T=None, max_corr_dist: float = 0.05, max_iter: int = 30,
               eps: float = 0.0, normal_radius: float = 0.1, normal_max_nn: int = 30) -> int:
        s, ns = self._host(src, "src")
        t, nt = self._host(tgt, "tgt")
        n, nn = self._host(tgt_nrm, "tgt_nrm")
        if tgt_nrm is not None and nn != nt:
            raise O3GError(ERR_ARG, "o3g_server_submit", "normals must match the target points one to one")
        T0 = _pose(np.eye(4) if init_T is None else init_T)
        rid = _i64()
        _check(lib().o3g_server_submit(self._h, _vp(s.ctypes.data if ns else 0), ns, _vp(t.ctypes.data if nt else 0),
                                       nt, _vp(n.ctypes.data) if n is not None and nn else _vp(0),
                                       float(normal_radius), int(normal_max_nn), _pp(T0), float(max_corr_dist),
                                       int(max_iter), float(eps), ctypes.byref(rid)), "o3g_server_submit")
        return rid.value

    def step(self):
        """One scheduling step; returns (active, waiting, completed_this_step)."""
        a, w, c = _i32(), _i32(), _i32()
        _check(lib().o3g_server_step(self._h, ctypes.byref(a), ctypes.byref(w), ctypes.byref(c)), "o3g_server_step")
        return a.value, w.value, c.value

    def completed(self, cap: int = 4096) -> list:
        """Ids of finished requests not yet polled."""
        ids = np.zeros(cap, np.int64)
        n = _i32()
        _check(lib().o3g_server_completed(self._h, ids.ctypes.data_as(_vp), int(cap), ctypes.byref(n)),
               "o3g_server_completed")
        return ids[: n.value].tolist()

    def poll(self, rid: int):
        """The result dict of a finished request (then forgotten), or None while it is in flight."""
        done, st, iters = _i32(), _i32(), _i32()
        T = np.zeros(16)
        fit, rmse = _f64(), _f64()
        _check(lib().o3g_server_poll(self._h, int(rid), ctypes.byref(done), _pp(T), ctypes.byref(fit),
                                     ctypes.byref(rmse), ctypes.byref(iters), ctypes.byref(st)), "o3g_server_poll")
        if not done.value:
            return None
        return dict(status=st.value, T=T.reshape(4, 4), fitness=fit.value, rmse=rmse.value, iters=iters.value)


def icp_point_to_plane(src, tgt, tgt_nrm, init_T, max_corr_dist: float, max_iter: int) -> dict:
    """One-shot point-to-plane ICP on device clouds (builds and frees the target grid)."""
    _torch().cuda.synchronize()
    ps, ns, ss = _cloud(src, "src")
    pt, nt, stt = _cloud(tgt, "tgt")
    pn, nn, sn = _cloud(tgt_nrm, "tgt_nrm")
    T0 = _pose(init_T)
    T = np.zeros(16)
    fit, rmse = _f64(), _f64()
    st = _check(lib().o3g_icp_point_to_plane(ps, ns, ss, pt, nt, stt, pn, nn, sn, _pp(T0), float(max_corr_dist),
                                             int(max_iter), _pp(T), ctypes.byref(fit), ctypes.byref(rmse)),
                "o3g_icp_point_to_plane")
    return _result(st, T, fit, rmse, None)


def register_point_to_plane(src, tgt, tgt_nrm, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                            normal_radius: float = 0.1, normal_max_nn: int = 30, stream=None) -> dict:
    """Whole refinement from device clouds (o3g_register_point_to_plane): target grid, target normals
    (attached `tgt_nrm`, or estimated with (normal_radius, normal_max_nn) when None), ICP; the source's
    sort runs beside the grid build and the normals.  Returns dict(status, T, fitness, rmse, iters)."""
    ps, ns, ss = _cloud(src, "src")
    pt, nt, st_ = _cloud(tgt, "tgt")
    if tgt_nrm is not None:
        pn, nn, sn = _cloud(tgt_nrm, "tgt_nrm")
        if nn != nt:
            raise O3GError(ERR_ARG, "register_point_to_plane", "normals must match the target points one to one")
    else:
        pn, sn = _vp(0), 3
    T0 = _pose(init_T)
    T = np.zeros(16)
    fit, rmse, iters = _f64(), _f64(), _i32()
    st = _check(lib().o3g_register_point_to_plane(ps, ns, ss, pt, nt, st_, pn, sn, float(normal_radius),
                                                  int(normal_max_nn), _pp(T0), float(max_corr_dist), int(max_iter),
                                                  float(eps), _pp(T), ctypes.byref(fit), ctypes.byref(rmse),
                                                  ctypes.byref(iters), _stream(stream)),
                "o3g_register_point_to_plane")
    return _result(st, T, fit, rmse, iters)


def register_point_to_plane_host(src, tgt, tgt_nrm, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                                 normal_radius: float = 0.1, normal_max_nn: int = 30, stream=None) -> dict:
    """Whole refinement from host arrays (N x 3 float32, C-contiguous; page-locked tensors copy asynchronously).

    `src`, `tgt`, `tgt_nrm` may be numpy arrays or CPU torch tensors; `tgt_nrm=None`
    estimates the target normals on the GPU with (normal_radius, normal_max_nn).
    """
    def host_ptr(a, name):
        if a is None:
            return _vp(0), 0
        torch = _torch()
        if isinstance(a, torch.Tensor):
            if a.is_cuda or a.dtype != torch.float32 or not a.is_contiguous() or (a.numel() and a.shape[-1] != 3):
                raise TypeError(f"{name} must be a contiguous N x 3 float32 host tensor")
            return _vp(a.data_ptr() if a.numel() else 0), a.shape[0]
        arr = np.asarray(a)
        if arr.dtype != np.float32 or not arr.flags.c_contiguous or (arr.size and arr.shape[-1] != 3):
            raise TypeError(f"{name} must be a C-contiguous N x 3 float32 array")
        return _vp(arr.ctypes.data if arr.size else 0), arr.shape[0] if arr.ndim == 2 else 0

    ps, ns = host_ptr(src, "src")
    pt, nt = host_ptr(tgt, "tgt")
    pn, nn = host_ptr(tgt_nrm, "tgt_nrm")
    if tgt_nrm is not None and nn != nt:
        raise O3GError(ERR_ARG, "register_point_to_plane_host", "normals must match the target points one to one")
    T0 = _pose(init_T)
    T = np.zeros(16)
    fit, rmse, iters = _f64(), _f64(), _i32()
    st = _check(lib().o3g_register_point_to_plane_host(ps, ns, pt, nt, pn, float(normal_radius), int(normal_max_nn),
                                                       _pp(T0), float(max_corr_dist), int(max_iter), float(eps),
                                                       _pp(T), ctypes.byref(fit), ctypes.byref(rmse),
                                                       ctypes.byref(iters), _stream(stream)),
                "o3g_register_point_to_plane_host")
    return _result(st, T, fit, rmse, iters)
