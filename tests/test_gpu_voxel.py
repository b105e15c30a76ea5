"""Voxel downsampling on the GPU (voxel_down_sample, Sec. 3.1 / Fig. 1) against the oracle, bit for bit.

Both sides take the voxel index from one correctly rounded float32 division,
order voxels by (ix, iy, iz) and sum each voxel's points in float64 in input
order, so centroids and counts must agree exactly.
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


def check(o3g, p, v):
    c, cnt = o3g.voxel_down_sample(cuda(p), v, with_counts=True)
    c_ref, cnt_ref = oracle.voxel_down_sample(p, v)
    assert np.array_equal(cnt.cpu().numpy(), cnt_ref)
    assert np.array_equal(c.cpu().numpy(), c_ref)
    return len(c_ref)


@pytest.mark.parametrize("n,v,span", [(50000, 0.05, 1.0), (20000, 0.007, 0.2), (3000, 10.0, 1.0),
                                      (100000, 0.002, 1.0), (7, 0.1, 1.0)])
def test_voxel_bitexact_random(o3g, n, v, span):
    g = synth.rng(600 + n)
    p = g.uniform(-span, span, (n, 3)).astype(np.float32)
    if n > 10:
        p[: n // 10] = (np.round(p[: n // 10] / np.float32(v)) * np.float32(v)).astype(np.float32)
        p[n // 10: n // 5] = p[: n // 10]
    m = check(o3g, p, v)
    assert 0 < m <= n


def test_voxel_wide_extent_uses_the_multi_pass_order(o3g):
    """Extents needing more than 31 key bits (sparse far points with a fine voxel) go through the per-axis
    passes; the result is still the oracle's."""
    g = synth.rng(610)
    p = np.concatenate([g.uniform(-1, 1, (20000, 3)), g.uniform(-3000, 3000, (500, 3))]).astype(np.float32)
    check(o3g, p, 0.004)


def test_voxel_raw_rgbd_frame(o3g):
    """A raw 640x480 ray-cast frame (~300k points) thinned at 0.01 m, the generator's workload, at full size."""
    g = synth.rng(2)
    room = synth.make_room(g)
    pts = synth.back_project(synth.depth_frame(room, np.eye(4), g)).astype(np.float32)
    m = check(o3g, pts, 0.01)
    assert 50000 < m < 150000


def test_voxel_edge_cases(o3g):
    import torch
    empty = o3g.voxel_down_sample(torch.zeros((0, 3), device="cuda"), 0.1)
    assert empty.shape[0] == 0
    p = np.array([[0, 0, 0], [np.nan, 0, 0], [0.01, 0.02, 0.03], [np.inf, 1, 1], [0.5, 0.5, 0.5]], np.float32)
    check(o3g, p, 0.1)
    allbad = np.full((5, 3), np.nan, np.float32)
    assert o3g.voxel_down_sample(cuda(allbad), 0.1).shape[0] == 0
    with pytest.raises(o3g.O3GError):
        o3g.voxel_down_sample(cuda(np.array([[1e9, 0, 0]], np.float32)), 0.1)
    with pytest.raises(o3g.O3GError):
        o3g.voxel_down_sample(cuda(p), -1.0)
    # strided rows (x, y, z, extra)
    g = synth.rng(611)
    q = g.uniform(-1, 1, (5000, 4)).astype(np.float32)
    c = o3g.voxel_down_sample(cuda(q), 0.1)
    c_ref, _ = oracle.voxel_down_sample(np.ascontiguousarray(q[:, :3]), 0.1)
    assert np.array_equal(c.cpu().numpy(), c_ref)
