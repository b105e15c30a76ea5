"""Hypothesis validation on the GPU (RANSAC's check of candidate poses, Sec. 3.3) against the oracle.

Inlier counts and fitness are exact (the correspondences are bit-exact), the
inlier rmse agrees to float64 summation-order rounding.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from paper_1801_09847_gb300 import synth

pytestmark = pytest.mark.gpu


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


def hypotheses(g, count, T_gt):
    """Candidate poses as RANSAC draws them: mostly wrong, a few near the truth, one exact."""
    out = [T_gt]
    for k in range(count - 1):
        if k % 10 == 0:
            out.append(synth.perturbation(g, 0.5, 0.005) @ T_gt)
        else:
            out.append(synth.perturbation(g, float(g.uniform(2, 60)), float(g.uniform(0.02, 0.5))) @ T_gt)
    return out


def check(o3g, grid, src, tgt, poses, r, method="brute"):
    fit, rmse, cnt = o3g.evaluate_poses(grid, cuda(src), poses, r)
    f_ref, r_ref, c_ref = oracle.evaluate_poses(src, tgt, poses, r, nn_method=method)
    assert np.array_equal(cnt, c_ref)
    assert np.array_equal(fit, f_ref)
    assert np.allclose(rmse, r_ref, rtol=1e-12, atol=0)
    return fit


def test_evaluate_sphere_plane_many_hypotheses(o3g):
    pr = synth.sphere_plane_pair()
    grid = o3g.build_grid(cuda(pr.tgt), 0.05 * 1.002)
    poses = hypotheses(synth.rng(130), 200, pr.T_gt)
    fit = check(o3g, grid, pr.src, pr.tgt, poses, 0.05)
    assert fit[0] > 0.95 and fit[0] > np.median(fit)


def test_evaluate_room_frame_full_size(o3g):
    """The RGB-D frame pair at full size (94,829 sources), 40 hypotheses, grid oracle."""
    pr = synth.room_frame_pair()
    grid = o3g.build_grid(cuda(pr.tgt), 0.05 * 1.002)
    poses = hypotheses(synth.rng(131), 40, pr.T_gt)
    check(o3g, grid, pr.src, pr.tgt, poses, 0.05, method="grid")


@pytest.mark.parametrize("cell_factor", [0.5, 1.0, 2.0])
def test_evaluate_cell_sizes(o3g, cell_factor):
    g = synth.rng(132)
    tgt = g.uniform(-1, 1, (5000, 3)).astype(np.float32)
    src = (tgt[g.integers(0, 5000, 3000)] + g.normal(0, 0.02, (3000, 3))).astype(np.float32)
    grid = o3g.build_grid(cuda(tgt), 0.08 * cell_factor)
    check(o3g, grid, src, tgt, hypotheses(g, 30, np.eye(4)), 0.08)


def test_evaluate_edge_cases(o3g):
    pr = synth.sphere_plane_pair(n=500)
    grid = o3g.build_grid(cuda(pr.tgt), 0.05)
    fit, rmse, cnt = o3g.evaluate_poses(grid, cuda(pr.src), np.zeros((0, 4, 4)), 0.05)
    assert len(fit) == 0
    import torch
    fit, rmse, cnt = o3g.evaluate_poses(grid, torch.zeros((0, 3), device="cuda"), [np.eye(4)], 0.05)
    assert fit[0] == 0.0 and rmse[0] == 0.0 and cnt[0] == 0
    far = synth.make_T(np.eye(3), [10.0, 0.0, 0.0])
    fit, rmse, cnt = o3g.evaluate_poses(grid, cuda(pr.src), [far], 0.05)
    assert fit[0] == 0.0 and rmse[0] == 0.0
    bad = np.eye(4)
    bad[0, 3] = np.nan
    with pytest.raises(o3g.O3GError):
        o3g.evaluate_poses(grid, cuda(pr.src), [bad], 0.05)
