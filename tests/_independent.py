"""Independent numpy/scipy computations used to pin the oracle.

Nothing here imports the oracle or the CUDA library.  Each routine is a
different route to a quantity the paper or the mathematics fixes, so that a
mistake in the oracle (a dropped term, a wrong sign, a transposed operand)
shows up as a disagreement.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg


def nn_bruteforce_f32(p, tgt, r_max):
    """Fixed-radius NN with numpy FP32 elementwise arithmetic; lowest index on ties."""
    p = np.asarray(p, np.float32)
    tgt = np.asarray(tgt, np.float32)
    r2 = np.float32(r_max) * np.float32(r_max)
    corr = np.full(len(p), -1, np.int32)
    d2o = np.zeros(len(p), np.float32)
    if len(tgt) == 0:
        return corr, d2o
    for i in range(len(p)):
        d = p[i][None, :] - tgt  # float32
        d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
        ok = d2 <= r2
        if ok.any():
            m = d2[ok].min()
            j = np.flatnonzero(ok & (d2 == m))[0]
            corr[i] = j
            d2o[i] = d2[j]
    return corr, d2o


def knn_bruteforce_f32(pts, q, radius, max_nn):
    """Hybrid kNN for one query with numpy FP32 arithmetic: indices sorted by (d2, index)."""
    pts = np.asarray(pts, np.float32)
    d = np.asarray(q, np.float32)[None, :] - pts
    d2 = (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]
    r2 = np.float32(radius) * np.float32(radius)
    idx = np.flatnonzero(d2 <= r2)
    order = np.lexsort((idx, d2[idx]))
    return idx[order][:max_nn], d2[idx][order][:max_nn]


def skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]], np.float64)


def se3_exp_left(xi, p):
    """exp([w]x) p + v in FP64 via scipy's matrix exponential (a route independent of any Euler formula)."""
    R = scipy.linalg.expm(skew(xi[:3]))
    return np.asarray(p, np.float64) @ R.T + np.asarray(xi[3:], np.float64)


def residuals(xi, p, q, n):
    """Point-to-plane residuals r_i(xi) = (exp(xi) p_i - q_i) . n_i in FP64."""
    return np.sum((se3_exp_left(xi, p) - np.asarray(q, np.float64)) * np.asarray(n, np.float64), axis=1)


def fd_jacobian(p, q, n, h=1e-6):
    """Central finite-difference Jacobian of the stacked residual vector at xi = 0 (N x 6)."""
    J = np.empty((len(p), 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        J[:, k] = (residuals(e, p, q, n) - residuals(-e, p, q, n)) / (2 * h)
    return J
