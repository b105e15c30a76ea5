"""Precision study on the GPU: float32 terms with compensated block sums against all-float64 terms.

The 2M-point scene-fragment pair (two fused 50-frame fragments of one room,
0.005 m voxels, max_correspondence_distance 0.02, 50 iterations) is the
full-size case; the oracle answers its correspondence step through the exact
grid search (pinned bit-exact to the brute-force scan in test_oracle_pins.py)
and is anchored here once more to the scan on a seeded sample.  Both GPU
precisions must give the oracle's correspondences bit for bit, its normal
equations within the stated bars, and its final pose within 1e-6 rad / 1e-6 m.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1801_09847_gb300 import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-6
F32_TOL = 1e-5   # relative error of J^T J (Frobenius) and of J^T r (scaled), float32 terms
F64_TOL = 1e-11  # float64 terms equal the oracle's; only the summation order differs (n eps at worst)


@pytest.fixture(scope="module")
def o3g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09847_gb300 import build, o3g as mod
    build.build()
    oracle.build()
    mod.lib()
    return mod


def cuda(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def equations_ref(src, tgt, nrm, T, r):
    """The oracle's normal equations at pose T (grid search), plus the scale sum_i |J_i| |r_i| of J^T r."""
    p = oracle.transform(src, T)
    corr, d2 = oracle.nn(p, tgt, r, method="grid")
    A, b, sr2, sd2, cnt = oracle.normal_equations(p, tgt, nrm, corr, d2)
    m = corr >= 0
    pp = p[m].astype(np.float64)
    q = tgt[corr[m]].astype(np.float64)
    n = nrm[corr[m]].astype(np.float64)
    J = np.hstack([np.cross(pp, n), n])
    res = np.sum((pp - q) * n, axis=1)
    return A, b, np.array([sr2, sd2, cnt]), np.abs(J).T @ np.abs(res), corr, d2


def errors(A, b, A_ref, b_ref, scale_b):
    return np.linalg.norm(A - A_ref) / np.linalg.norm(A_ref), np.max(np.abs(b - b_ref)) / np.max(scale_b)


@pytest.mark.parametrize("which", ["sphere_plane", "corner"])
def test_f64_normal_equations_small(o3g, which):
    """Small clouds, several poses: float64 terms agree with the oracle to summation-order rounding."""
    if which == "sphere_plane":
        pr = synth.sphere_plane_pair()
        src, tgt, nrm, r = pr.src, pr.tgt, pr.tgt_nrm, pr.max_corr_dist
        Ts = [np.eye(4), pr.T_gt]
    else:
        g = synth.rng(31)
        ax = np.arange(0.0, 1.0, 0.02)
        u, v = [a.ravel() for a in np.meshgrid(ax, ax)]
        z = np.zeros_like(u)
        tgt = np.concatenate([np.stack([u, v, z], 1), np.stack([u, z, v], 1), np.stack([z, u, v], 1)])
        nrm = np.concatenate([np.tile([0, 0, 1.0], (len(u), 1)), np.tile([0, 1.0, 0], (len(u), 1)),
                              np.tile([1.0, 0, 0], (len(u), 1))]).astype(np.float32)
        tgt = (tgt + g.normal(0, 0.002, tgt.shape)).astype(np.float32)
        src = synth.apply_T(np.linalg.inv(synth.perturbation(g, 3.0, 0.02)), tgt).astype(np.float32)
        r = 0.05
        Ts = [np.eye(4), synth.perturbation(g, 1.0, 0.01)]
    grid = o3g.build_grid(cuda(tgt), r * 1.002)
    grid.set_normals(cuda(nrm))
    for T in Ts:
        A_ref, b_ref, st_ref, scale_b, _, _ = equations_ref(src, tgt, nrm, T, r)
        A64, b64, st64 = o3g.normal_equations(grid, cuda(src), T, r, precision="f64")
        A32, b32, _ = o3g.normal_equations(grid, cuda(src), T, r, precision="f32")
        ea64, eb64 = errors(A64, b64, A_ref, b_ref, scale_b)
        ea32, eb32 = errors(A32, b32, A_ref, b_ref, scale_b)
        assert ea64 <= F64_TOL and eb64 <= F64_TOL, (ea64, eb64)
        assert ea32 <= F32_TOL and eb32 <= F32_TOL, (ea32, eb32)
        assert np.array_equal(A64, A64.T)
        assert st64[2] == st_ref[2]
        assert st64[1] == pytest.approx(st_ref[1], rel=1e-12)
        assert st64[0] == pytest.approx(st_ref[0], rel=1e-11, abs=1e-300)


def test_f64_icp_small_matches_oracle(o3g):
    """All-float64 ICP on the noise-free corner is the oracle's registration within 1e-6, like float32."""
    g = synth.rng(32)
    ax = np.arange(0.0, 1.0, 0.02)
    u, v = [a.ravel() for a in np.meshgrid(ax, ax)]
    z = np.zeros_like(u)
    tgt = np.concatenate([np.stack([u, v, z], 1), np.stack([u, z, v], 1), np.stack([z, u, v], 1)]).astype(np.float32)
    nrm = np.concatenate([np.tile([0, 0, 1.0], (len(u), 1)), np.tile([0, 1.0, 0], (len(u), 1)),
                          np.tile([1.0, 0, 0], (len(u), 1))]).astype(np.float32)
    T_gt = synth.perturbation(g, 2.0, 0.02)
    src = synth.apply_T(np.linalg.inv(T_gt), tgt).astype(np.float32)
    grid = o3g.build_grid(cuda(tgt), 0.05 * 1.002)
    grid.set_normals(cuda(nrm))
    ref = oracle.icp_point_to_plane(src, tgt, nrm, np.eye(4), 0.05, 20)
    for prec in ("f32", "f64"):
        res = o3g.icp_point_to_plane_grid(grid, cuda(src), np.eye(4), 0.05, 20, precision=prec)
        assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
        ang, dt = synth.pose_error(res["T"], ref["T"])
        assert ang <= POSE_TOL and dt <= POSE_TOL, (prec, ang, dt)


def test_precision_argument_validated(o3g):
    tgt = np.zeros((10, 3), np.float32)
    grid = o3g.build_grid(cuda(tgt), 0.1)
    grid.set_normals(cuda(np.tile(np.float32([0, 0, 1]), (10, 1))))
    with pytest.raises(ValueError):
        o3g.normal_equations(grid, cuda(tgt), np.eye(4), 0.1, precision="f16")
    T, A, b, stats = np.eye(4).ravel().copy(), np.zeros(36), np.zeros(6), np.zeros(3)
    st = o3g.lib().o3g_normal_equations_ex(grid.handle, None, 0, 3, o3g._pp(T), 0.1, 7, o3g._pp(A), o3g._pp(b),
                                           o3g._pp(stats), None)
    assert st == o3g.ERR_ARG


# ----------------------------------------------------------- the 2M-point fragment pair


@pytest.fixture(scope="module")
def frag(o3g):
    pr = synth.fragment_pair()
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist * 1.002)
    grid.set_normals(cuda(pr.tgt_nrm))
    return pr, grid, cuda(pr.src)


@pytest.fixture(scope="module")
def frag_oracle(frag):
    pr = frag[0]
    return oracle.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter,
                                     nn_method="grid")


def test_fragment_correspondences_bitexact(o3g, frag, frag_oracle):
    """All 2M correspondences bit-exact at the start pose and at the oracle's final pose; a seeded sample is
    also checked against the brute-force scan itself."""
    pr, grid, src = frag
    for T in (np.eye(4), frag_oracle["T"]):
        corr, d2 = o3g.correspondences(grid, src, T, pr.max_corr_dist)
        corr, d2 = corr.cpu().numpy(), d2.cpu().numpy()
        p = oracle.transform(pr.src, T)
        c_ref, d_ref = oracle.nn(p, pr.tgt, pr.max_corr_dist, method="grid")
        assert np.array_equal(corr, c_ref) and np.array_equal(d2, d_ref)
        idx = np.sort(synth.rng(33).choice(len(p), 1024, replace=False))
        c_bf, d_bf = oracle.nn(p[idx], pr.tgt, pr.max_corr_dist)
        assert np.array_equal(corr[idx], c_bf) and np.array_equal(d2[idx], d_bf)


def test_fragment_normal_equations_both_precisions(o3g, frag, frag_oracle):
    pr, grid, src = frag
    for T in (np.eye(4), frag_oracle["T"]):
        A_ref, b_ref, st_ref, scale_b, _, _ = equations_ref(pr.src, pr.tgt, pr.tgt_nrm, T, pr.max_corr_dist)
        A32, b32, st32 = o3g.normal_equations(grid, src, T, pr.max_corr_dist, precision="f32")
        A64, b64, st64 = o3g.normal_equations(grid, src, T, pr.max_corr_dist, precision="f64")
        ea32, eb32 = errors(A32, b32, A_ref, b_ref, scale_b)
        ea64, eb64 = errors(A64, b64, A_ref, b_ref, scale_b)
        assert ea32 <= F32_TOL and eb32 <= F32_TOL, (ea32, eb32)
        assert ea64 <= F64_TOL and eb64 <= F64_TOL, (ea64, eb64)
        assert st32[2] == st_ref[2] and st64[2] == st_ref[2]


def test_fragment_icp_both_precisions_within_1e6(o3g, frag, frag_oracle):
    """50 iterations on 2M points: both precisions end within 1e-6 rad / 1e-6 m of the oracle's pose, with its
    iteration count and status; fitness equals the oracle's evaluation at the GPU's own final pose."""
    pr, grid, src = frag
    ref = frag_oracle
    assert ref["fitness"] > 0.9
    for prec in ("f32", "f64"):
        res = o3g.icp_point_to_plane_grid(grid, src, np.eye(4), pr.max_corr_dist, pr.max_iter, precision=prec)
        assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
        ang, dt = synth.pose_error(res["T"], ref["T"])
        assert ang <= POSE_TOL and dt <= POSE_TOL, (prec, ang, dt)
        assert abs(res["fitness"] - ref["fitness"]) <= 1e-5


def test_fragment_warm_search_correspondence_set_bitexact(o3g, frag):
    """The correspondence set of the final evaluation (found by the warm-started search of the iterations:
    before candidate lists, the grid search from the previous matches; then each point's list where it still
    covers the point, the grid search and a rebuilt list where it does not) after 1, 3, 11 (lists just built),
    20 (lists being rebuilt as points drift) and 50 iterations: all 2M matches bit-exact against the oracle's
    search at the GPU's own final pose."""
    pr, grid, src = frag
    for k in (1, 3, 11, 20, pr.max_iter):
        res = o3g.icp_point_to_plane_grid(grid, src, np.eye(4), pr.max_corr_dist, k, correspondences=True)
        p = oracle.transform(pr.src, res["T"])
        c_ref, d_ref = oracle.nn(p, pr.tgt, pr.max_corr_dist, method="grid")
        assert np.array_equal(res["corr"].cpu().numpy(), c_ref), k
        assert np.array_equal(res["d2"].cpu().numpy(), d_ref), k
        assert res["fitness"] == float(np.count_nonzero(c_ref >= 0)) / len(c_ref)
