"""Point-to-point ICP on the GPU (TransformationEstimationPointToPoint, Sec. 3.3) against the oracle.

The GPU solves Horn's quaternion problem by Newton's method on the
characteristic quartic of the scaled 4x4 and an adjugate column; the oracle
diagonalises the same 4x4 by cyclic Jacobi and is itself pinned against an SVD
Kabsch solution (test_oracle_pins.py).  Checks: every GPU iterate is the
oracle's closed-form step from the GPU's previous iterate (within 1e-7), the
end-to-end pose within 1e-6 rad / 1e-6 m where the problem is well conditioned,
statuses, and fitness / rmse at the final pose.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1801_09847_gb300 import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-6
SHADOW_TOL = 1e-7


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


def oracle_step(src, tgt, T, r, method="brute"):
    p = oracle.transform(src, T)
    corr, _ = oracle.nn(p, tgt, r, method=method)
    dT, deg, _, cnt = oracle.rigid_align(p, tgt, corr)
    return dT @ T, deg, cnt


def shadow(o3g, grid, src, tgt, r, K, method="brute"):
    worst = 0.0
    T = np.eye(4)
    for k in range(1, K + 1):
        res = o3g.icp_point_to_point_grid(grid, cuda(src), np.eye(4), r, k)
        T_next, _, _ = oracle_step(src, tgt, T, r, method)
        ang, dt = synth.pose_error(res["T"], T_next)
        worst = max(worst, ang, dt)
        assert ang <= SHADOW_TOL and dt <= SHADOW_TOL, (k, ang, dt)
        T = res["T"]
    return T, worst


def test_p2p_sphere_plane_shadows_oracle(o3g):
    pr = synth.sphere_plane_pair(deg=3.0, trans=0.02)
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist * 1.002)
    shadow(o3g, grid, pr.src, pr.tgt, pr.max_corr_dist, 12)
    res = o3g.icp_point_to_point_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, 30)
    ev = oracle.icp_point_to_point(pr.src, pr.tgt, res["T"], pr.max_corr_dist, 0)
    assert res["fitness"] == ev["fitness"]
    assert res["rmse"] == pytest.approx(ev["rmse"], rel=1e-6)


def test_p2p_noise_free_end_to_end_within_1e6(o3g):
    """Noise-free sphere-plus-plane: GPU and oracle both reach the ground truth and each other within 1e-6."""
    pr = synth.sphere_plane_pair(noise=0.0, deg=3.0, trans=0.02)
    grid = o3g.build_grid(cuda(pr.tgt), 0.05 * 1.002)
    res = o3g.icp_point_to_point_grid(grid, cuda(pr.src), np.eye(4), 0.05, 200, eps=1e-9)
    ref = oracle.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 200, eps=1e-9)
    assert res["status"] == ref["status"] == o3g.OK
    for T in (ref["T"], pr.T_gt):
        ang, dt = synth.pose_error(res["T"], T)
        assert ang <= 1e-5 and dt <= 1e-5, (ang, dt)
    ang, dt = synth.pose_error(res["T"], ref["T"])
    assert ang <= POSE_TOL and dt <= POSE_TOL, (ang, dt)
    assert res["fitness"] == 1.0


def test_p2p_room_frame_shadows_oracle(o3g):
    pr = synth.room_frame_pair()
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist * 1.002)
    g = synth.rng(41)
    src = pr.src[np.sort(g.choice(len(pr.src), 30000, replace=False))]
    shadow(o3g, grid, src, pr.tgt, pr.max_corr_dist, 6, method="grid")


def test_p2p_statuses(o3g):
    # collinear target: the rotation is undetermined -> degenerate, pure translation
    t = np.linspace(-1, 1, 400, dtype=np.float32)
    line = np.stack([t, 0.5 * t, -t], 1).astype(np.float32)
    grid = o3g.build_grid(cuda(line), 0.05)
    src = (line + np.float32([0.01, 0.0, 0.0])).astype(np.float32)
    res = o3g.icp_point_to_point_grid(grid, cuda(src), np.eye(4), 0.05, 3)
    ref = oracle.icp_point_to_point(src, line, np.eye(4), 0.05, 3)
    assert res["status"] == ref["status"] == o3g.WARN_DEGENERATE
    assert np.array_equal(res["T"][:3, :3], np.eye(3))
    assert np.allclose(res["T"], ref["T"], atol=1e-9)
    # no partners at all
    far = o3g.icp_point_to_point_grid(grid, cuda(src + np.float32(5)), np.eye(4), 0.05, 3)
    assert far["status"] == o3g.WARN_FEW_CORR and far["iters"] == 0 and far["fitness"] == 0.0
    # eps stop matches the oracle's iteration count on a well-conditioned pair
    pr = synth.sphere_plane_pair(n=3000, noise=0.0, deg=2.0, trans=0.01)
    grid = o3g.build_grid(cuda(pr.tgt), 0.05 * 1.002)
    a = o3g.icp_point_to_point_grid(grid, cuda(pr.src), np.eye(4), 0.05, 300, eps=1e-6)
    b = oracle.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 300, eps=1e-6)
    assert a["iters"] < 300 and abs(a["iters"] - b["iters"]) <= 1


def test_p2p_far_from_origin(o3g):
    """Clouds 100 m from the origin: the moments are taken about the grid centre, so FP32 terms keep their
    precision and the GPU still shadows the oracle."""
    pr = synth.sphere_plane_pair(n=3000, deg=3.0, trans=0.02)
    off = np.float32([100.0, -50.0, 30.0])
    tgt = (pr.tgt + off).astype(np.float32)
    src = (pr.src + off).astype(np.float32)
    grid = o3g.build_grid(cuda(tgt), 0.05 * 1.002)
    shadow(o3g, grid, src, tgt, 0.05, 5)
