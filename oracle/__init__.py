"""CPU oracle for point-to-plane ICP and hybrid-kNN PCA normals (Open3D, arXiv 1801.09847).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference legs of ``bench.py`` import this package.  The CUDA
library never links, loads or calls it, and it shares no code with it.

The arithmetic lives in ``o3g_oracle.c`` (plain C, FP64 accumulation, compiled
with ``-ffp-contract=off`` so each FP32 expression is a chain of separately
rounded IEEE operations).  This module only compiles it with gcc and marshals
numpy arrays through ctypes.  Every function cites the passage of the paper
it follows; see the header of ``o3g_oracle.c`` for the readings taken where the
paper is silent.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "o3g_oracle.c")
_LIB = os.path.join(_HERE, "_o3g_oracle.so")
_lock = threading.Lock()
_lib = None

OK, WARN_DEGENERATE, WARN_FEW_CORR, ERR_ARG, ERR_OOM = 0, 1, 2, -1, -2

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_i32 = ctypes.c_int32


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (idempotent)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
               "-pthread", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build())
    lib.ora_transform.argtypes = [_f32p, _i64, _f64p, _f32p]
    lib.ora_transform.restype = None
    lib.ora_nn.argtypes = [_f32p, _i64, _f32p, _i64, ctypes.c_float, _i32, _i32p, _f32p]
    lib.ora_nn.restype = ctypes.c_int
    lib.ora_normal_equations.argtypes = [_f32p, _i64, _f32p, _f32p, _i32p, _f32p, _f64p, _f64p,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_int64)]
    lib.ora_normal_equations.restype = None
    lib.ora_residual_jacobian.argtypes = [_f32p, _f32p, _f32p, _f64p, ctypes.POINTER(ctypes.c_double)]
    lib.ora_residual_jacobian.restype = None
    lib.ora_ldlt_solve.argtypes = [_f64p, _f64p, _f64p]
    lib.ora_ldlt_solve.restype = ctypes.c_int
    lib.ora_delta_T.argtypes = [_f64p, _f64p]
    lib.ora_delta_T.restype = None
    lib.ora_mat4_mul.argtypes = [_f64p, _f64p, _f64p]
    lib.ora_mat4_mul.restype = None
    lib.ora_icp_point_to_plane.argtypes = [_f32p, _i64, _f32p, _i64, _f32p, _f64p, ctypes.c_double, _i32,
                                           ctypes.c_double, _i32, _f64p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    lib.ora_icp_point_to_plane.restype = ctypes.c_int
    lib.ora_icp_point_to_plane_gridnn.argtypes = lib.ora_icp_point_to_plane.argtypes
    lib.ora_icp_point_to_plane_gridnn.restype = ctypes.c_int
    lib.ora_grid_build.argtypes = [_f32p, _i64, ctypes.c_float]
    lib.ora_grid_build.restype = ctypes.c_void_p
    lib.ora_grid_free.argtypes = [ctypes.c_void_p]
    lib.ora_grid_free.restype = None
    lib.ora_grid_nn.argtypes = [ctypes.c_void_p, _f32p, _i64, _i32, _i32p, _f32p]
    lib.ora_grid_nn.restype = ctypes.c_int
    lib.ora_jacobi_eig4.argtypes = [_f64p, _f64p, _f64p]
    lib.ora_jacobi_eig4.restype = None
    lib.ora_rigid_align.argtypes = [_f32p, _i64, _f32p, _i32p, _f64p, ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(ctypes.c_int64)]
    lib.ora_rigid_align.restype = ctypes.c_int
    lib.ora_icp_point_to_point.argtypes = [_f32p, _i64, _f32p, _i64, _f64p, ctypes.c_double, _i32, ctypes.c_double,
                                           _i32, _i32, _f64p, ctypes.POINTER(ctypes.c_double),
                                           ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]
    lib.ora_icp_point_to_point.restype = ctypes.c_int
    lib.ora_voxel_downsample.argtypes = [_f32p, _i64, ctypes.c_float, _f32p, _i32p, ctypes.POINTER(ctypes.c_int64)]
    lib.ora_voxel_downsample.restype = ctypes.c_int
    lib.ora_evaluate_poses.argtypes = [_f32p, _i64, _f32p, _i64, _f64p, _i32, ctypes.c_double, _i32, _i32, _f64p,
                                       _f64p, np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")]
    lib.ora_evaluate_poses.restype = ctypes.c_int
    lib.ora_knn_hybrid.argtypes = [_f32p, _i64, _f32p, _i64, ctypes.c_float, _i32, _i32, _i32p, _f32p, _i32p]
    lib.ora_knn_hybrid.restype = ctypes.c_int
    lib.ora_jacobi_eig3.argtypes = [_f64p, _f64p, _f64p]
    lib.ora_jacobi_eig3.restype = None
    lib.ora_estimate_normals.argtypes = [_f32p, _i64, ctypes.c_float, _i32, _f64p, _i32, _f32p,
                                         ctypes.c_void_p]
    lib.ora_estimate_normals.restype = ctypes.c_int
    _lib = lib
    return lib


def default_threads() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return max(1, os.cpu_count() or 1)


def _pts(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float32)
    if a.size == 0:
        return np.zeros((0, 3), np.float32)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must be N x 3")
    return a


def _pose(T) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64).reshape(4, 4)
    return T


def transform(src, T) -> np.ndarray:
    """Step a3: p_i = R s_i + t in FP32, R and t rounded from the FP64 pose (Eq. 2 evaluates at x^k)."""
    src = _pts(src)
    out = np.empty_like(src)
    if len(src):
        _load().ora_transform(src, len(src), _pose(T).ravel(), out)
    return out


def nn(p, tgt, r_max: float, threads: int | None = None, method: str = "brute"):
    """Step a4: brute-force fixed-radius nearest neighbour, lowest index on ties.

    Follows registration_icp's max_correspondence_distance (Sec. 3.3).  Returns
    (corr int32[N], d2 float32[N]); corr = -1 where no target lies within r_max.
    method="grid" answers the same map through the exact 27-cell grid search of
    ``ora_grid_nn`` (pinned bit-exact against the scan); it needs r_max > 0.
    """
    p, tgt = _pts(p), _pts(tgt)
    corr = np.empty(len(p), np.int32)
    d2 = np.empty(len(p), np.float32)
    if len(p) == 0:
        return corr, d2
    if method == "grid":
        lib = _load()
        g = lib.ora_grid_build(tgt if len(tgt) else np.zeros((1, 3), np.float32), len(tgt),
                               ctypes.c_float(np.float32(r_max)))
        if not g:
            raise ValueError("ora_grid_build failed (r_max must be positive and finite)")
        try:
            st = lib.ora_grid_nn(g, p, len(p), threads or default_threads(), corr, d2)
        finally:
            lib.ora_grid_free(g)
        if st != OK:
            raise ValueError(f"ora_grid_nn status {st}")
        return corr, d2
    if method != "brute":
        raise ValueError(f"unknown NN method {method!r}")
    st = _load().ora_nn(p, len(p), tgt if len(tgt) else np.zeros((1, 3), np.float32), len(tgt),
                        ctypes.c_float(np.float32(r_max)), threads or default_threads(), corr, d2)
    if st != OK:
        raise ValueError(f"ora_nn status {st}")
    return corr, d2


def residual_jacobian(p, q, n):
    """r = (p - q) . n and J = [p x n ; n] in FP64 for one correspondence (Eq. 1-2 terms)."""
    J = np.empty(6, np.float64)
    r = ctypes.c_double()
    _load().ora_residual_jacobian(np.ascontiguousarray(p, np.float32), np.ascontiguousarray(q, np.float32),
                                  np.ascontiguousarray(n, np.float32), J, ctypes.byref(r))
    return J, r.value


def normal_equations(p, tgt, nrm, corr, d2):
    """Step a5: A = sum J J^T, b = sum J r (FP64, increasing i) plus sum r^2, sum d2, |C| (Sec. 4)."""
    p, tgt, nrm = _pts(p), _pts(tgt), _pts(nrm)
    corr = np.ascontiguousarray(corr, np.int32)
    d2 = np.ascontiguousarray(d2, np.float32)
    A = np.zeros(36, np.float64)
    b = np.zeros(6, np.float64)
    sr2, sd2, cnt = ctypes.c_double(), ctypes.c_double(), ctypes.c_int64()
    if len(p):
        _load().ora_normal_equations(p, len(p), tgt if len(tgt) else np.zeros((1, 3), np.float32),
                                     nrm if len(nrm) else np.zeros((1, 3), np.float32), corr, d2, A, b,
                                     ctypes.byref(sr2), ctypes.byref(sd2), ctypes.byref(cnt))
    return A.reshape(6, 6), b, sr2.value, sd2.value, cnt.value


def ldlt_solve(A, b):
    """Step a6: xi = -A^-1 b by LDL^T with the frozen-pivot rule (Eq. 2).  Returns (xi, n_frozen)."""
    xi = np.zeros(6, np.float64)
    nf = _load().ora_ldlt_solve(np.ascontiguousarray(A, np.float64).ravel(),
                                np.ascontiguousarray(b, np.float64).ravel(), xi)
    return xi, nf


def delta_T(xi):
    """Step a6: dT = [Rz(gamma) Ry(beta) Rx(alpha), t; 0 1] from xi = (alpha, beta, gamma, tx, ty, tz)."""
    out = np.zeros(16, np.float64)
    _load().ora_delta_T(np.ascontiguousarray(xi, np.float64), out)
    return out.reshape(4, 4)


def icp_point_to_plane(src, tgt, tgt_nrm, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                       threads: int | None = None, nn_method: str = "brute") -> dict:
    """registration_icp(..., TransformationEstimationPointToPlane()) (Sec. 3.3), steps a3..a7.

    Returns dict(status, T (4x4 FP64), fitness, rmse, iters).  nn_method="grid"
    takes the correspondences from the exact grid search (same result; for clouds
    too large to scan).
    """
    if nn_method not in ("brute", "grid"):
        raise ValueError(f"unknown NN method {nn_method!r}")
    src, tgt, tgt_nrm = _pts(src), _pts(tgt), _pts(tgt_nrm)
    if len(tgt_nrm) != len(tgt):
        raise ValueError("target normals must have as many records as target points (Sec. 3.1)")
    T = np.zeros(16, np.float64)
    fit, rmse, iters = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    one = np.zeros((1, 3), np.float32)
    lib = _load()
    fn = lib.ora_icp_point_to_plane_gridnn if nn_method == "grid" else lib.ora_icp_point_to_plane
    st = fn(src if len(src) else one, len(src), tgt if len(tgt) else one, len(tgt),
                                        tgt_nrm if len(tgt_nrm) else one, _pose(init_T).ravel(),
                                        float(max_corr_dist), int(max_iter), float(eps),
                                        threads or default_threads(), T, ctypes.byref(fit), ctypes.byref(rmse),
                                        ctypes.byref(iters))
    if st < 0:
        raise ValueError(f"ora_icp_point_to_plane status {st}")
    return dict(status=st, T=T.reshape(4, 4), fitness=fit.value, rmse=rmse.value, iters=iters.value)


def knn_hybrid(pts, queries, radius: float, max_nn: int, threads: int | None = None):
    """KDTreeSearchParamHybrid(radius, max_nn) search by brute force (Fig. 1): (idx, d2, count)."""
    pts, queries = _pts(pts), _pts(queries)
    nq = len(queries)
    idx = np.empty((nq, max_nn), np.int32)
    dd = np.empty((nq, max_nn), np.float32)
    cnt = np.empty(nq, np.int32)
    if nq == 0:
        return idx, dd, cnt
    st = _load().ora_knn_hybrid(pts if len(pts) else np.zeros((1, 3), np.float32), len(pts), queries, nq,
                                ctypes.c_float(np.float32(radius)), int(max_nn), threads or default_threads(),
                                idx.reshape(-1), dd.reshape(-1), cnt)
    if st != OK:
        raise ValueError(f"ora_knn_hybrid status {st}")
    return idx, dd, cnt


def jacobi_eig3(C):
    """Cyclic Jacobi eigen-decomposition of a symmetric 3x3 (FP64): (evals, V) with V[:, k] <-> evals[k]."""
    ev = np.zeros(3, np.float64)
    V = np.zeros(9, np.float64)
    _load().ora_jacobi_eig3(np.ascontiguousarray(C, np.float64).ravel(), ev, V)
    return ev, V.reshape(3, 3)


def estimate_normals(pts, radius: float, max_nn: int, viewpoint=(0.0, 0.0, 0.0), threads: int | None = None,
                     return_evals: bool = False):
    """estimate_normals(pc, KDTreeSearchParamHybrid(radius, max_nn)) (Fig. 1, Sec. 3.3) by brute force."""
    pts = _pts(pts)
    n = len(pts)
    out = np.empty((n, 3), np.float32)
    ev = np.empty((n, 3), np.float64)
    if n == 0:
        return (out, ev) if return_evals else out
    st = _load().ora_estimate_normals(pts, n, ctypes.c_float(np.float32(radius)), int(max_nn),
                                      np.ascontiguousarray(viewpoint, np.float64), threads or default_threads(),
                                      out, ev.ctypes.data_as(ctypes.c_void_p))
    if st != OK:
        raise ValueError(f"ora_estimate_normals status {st}")
    return (out, ev) if return_evals else out


def jacobi_eig4(C):
    """Cyclic Jacobi eigen-decomposition of a symmetric 4x4 (FP64): (evals, V) with V[:, k] <-> evals[k]."""
    ev = np.zeros(4, np.float64)
    V = np.zeros(16, np.float64)
    _load().ora_jacobi_eig4(np.ascontiguousarray(C, np.float64).ravel(), ev, V)
    return ev, V.reshape(4, 4)


def rigid_align(p, tgt, corr):
    """TransformationEstimationPointToPoint's step (Sec. 3.3): Horn's closed-form rigid motion taking the
    matched p_i onto q_corr(i).  Returns (dT 4x4, degenerate flag, rotation angle, |C|)."""
    p, tgt = _pts(p), _pts(tgt)
    corr = np.ascontiguousarray(corr, np.int32)
    dT = np.zeros(16, np.float64)
    ang, cnt = ctypes.c_double(), ctypes.c_int64()
    deg = _load().ora_rigid_align(p if len(p) else np.zeros((1, 3), np.float32), len(p),
                                  tgt if len(tgt) else np.zeros((1, 3), np.float32),
                                  corr if len(corr) else np.zeros(1, np.int32), dT, ctypes.byref(ang),
                                  ctypes.byref(cnt))
    return dT.reshape(4, 4), bool(deg), ang.value, cnt.value


def icp_point_to_point(src, tgt, init_T, max_corr_dist: float, max_iter: int, eps: float = 0.0,
                       threads: int | None = None, nn_method: str = "brute") -> dict:
    """registration_icp(..., TransformationEstimationPointToPoint()) (Sec. 3.3).

    Returns dict(status, T (4x4 FP64), fitness, rmse, iters).
    """
    if nn_method not in ("brute", "grid"):
        raise ValueError(f"unknown NN method {nn_method!r}")
    src, tgt = _pts(src), _pts(tgt)
    T = np.zeros(16, np.float64)
    fit, rmse, iters = ctypes.c_double(), ctypes.c_double(), ctypes.c_int32()
    one = np.zeros((1, 3), np.float32)
    st = _load().ora_icp_point_to_point(src if len(src) else one, len(src), tgt if len(tgt) else one, len(tgt),
                                        _pose(init_T).ravel(), float(max_corr_dist), int(max_iter), float(eps),
                                        threads or default_threads(), int(nn_method == "grid"), T,
                                        ctypes.byref(fit), ctypes.byref(rmse), ctypes.byref(iters))
    if st < 0:
        raise ValueError(f"ora_icp_point_to_point status {st}")
    return dict(status=st, T=T.reshape(4, 4), fitness=fit.value, rmse=rmse.value, iters=iters.value)


def voxel_down_sample(pts, voxel: float):
    """voxel_down_sample (Sec. 3.1, Fig. 1): per occupied voxel floor(p / v) (FP32 quotient) the FP64
    centroid of its points in input order, rounded to FP32; voxels in increasing (ix, iy, iz).
    Returns (centroids float32 [M, 3], counts int32 [M])."""
    pts = _pts(pts)
    out = np.empty((max(len(pts), 1), 3), np.float32)
    cnt = np.empty(max(len(pts), 1), np.int32)
    m = ctypes.c_int64()
    st = _load().ora_voxel_downsample(pts if len(pts) else np.zeros((1, 3), np.float32), len(pts),
                                      ctypes.c_float(np.float32(voxel)), out, cnt, ctypes.byref(m))
    if st != OK:
        raise ValueError(f"ora_voxel_downsample status {st}")
    return out[: m.value].copy(), cnt[: m.value].copy()


def evaluate_poses(src, tgt, poses, max_corr_dist: float, threads: int | None = None, nn_method: str = "brute"):
    """RANSAC's hypothesis validation (Sec. 3.3): for each 4x4 pose, fitness, inlier rmse and inlier count of the
    whole source against the target at that pose.  Returns (fitness [H], rmse [H], count [H])."""
    if nn_method not in ("brute", "grid"):
        raise ValueError(f"unknown NN method {nn_method!r}")
    src, tgt = _pts(src), _pts(tgt)
    P = np.ascontiguousarray(np.asarray(poses, np.float64).reshape(-1, 16))
    H = len(P)
    fit = np.zeros(max(H, 1))
    rmse = np.zeros(max(H, 1))
    cnt = np.zeros(max(H, 1), np.int64)
    one = np.zeros((1, 3), np.float32)
    st = _load().ora_evaluate_poses(src if len(src) else one, len(src), tgt if len(tgt) else one, len(tgt),
                                    P if H else np.zeros((1, 16)), H, float(max_corr_dist),
                                    threads or default_threads(), int(nn_method == "grid"), fit, rmse, cnt)
    if st != OK:
        raise ValueError(f"ora_evaluate_poses status {st}")
    return fit[:H], rmse[:H], cnt[:H]
