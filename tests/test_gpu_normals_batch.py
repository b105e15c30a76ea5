"""Batched normal estimation and batched hybrid kNN (both clouds of a pair, or many clouds, in one launch).

Every cloud must get bit for bit what the one-cloud call gives it (the same
warp routine runs on the same inputs), and the one-cloud calls are themselves
checked against the oracle in test_gpu_parity.py; one cloud of the batch is
checked against the oracle here as well.
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


def clouds():
    pr = synth.room_frame_pair()
    out = [pr.tgt, pr.src]  # both clouds of one pair
    for k, n in enumerate((0, 7, 3000, 20000, 45000)):
        out.append(synth.sphere_plane(n, synth.rng(700 + k))[0].astype(np.float32))
    return out


@pytest.mark.parametrize("max_nn", [30, 8, 48])
def test_normals_batch_equals_one_cloud_calls(o3g, max_nn):
    import torch
    pts = clouds()
    radius = [0.05, 0.05] + [0.1] * (len(pts) - 2)
    vps = np.array([[0.0, 0.0, 0.0]] * 2 + [[0.1, -0.2, 0.3]] * (len(pts) - 2), np.float32)
    grids_a = [o3g.build_grid(cuda(p), 0.06) for p in pts]
    grids_b = [o3g.build_grid(cuda(p), 0.06) for p in pts]
    outs = [torch.zeros((len(p), 3), device="cuda") for p in pts]
    o3g.estimate_normals_batch(grids_a, radius, max_nn, viewpoints=vps, outs=outs)
    for g, p, r, v, o in zip(grids_b, pts, radius, vps, outs):
        ref = g.estimate_normals(r, max_nn, viewpoint=tuple(float(x) for x in v))
        assert torch.equal(ref, o)
    # and the grids carry them: the point-to-plane step sees the same normal equations
    A1, b1, _ = o3g.normal_equations(grids_a[0], cuda(pts[1]), np.eye(4), 0.05)
    A2, b2, _ = o3g.normal_equations(grids_b[0], cuda(pts[1]), np.eye(4), 0.05)
    assert np.array_equal(A1, A2) and np.array_equal(b1, b2)


def test_normals_batch_one_cloud_against_oracle(o3g):
    import torch
    pts = clouds()
    grids = [o3g.build_grid(cuda(p), 0.06) for p in pts]
    outs = [torch.zeros((len(p), 3), device="cuda") for p in pts]
    o3g.estimate_normals_batch(grids, 0.1, 30, outs=outs)
    p = pts[4]
    n_gpu = outs[4].cpu().numpy()
    n_ref, ev = oracle.estimate_normals(p, 0.1, 30, return_evals=True)
    ok = (ev[:, 1] - ev[:, 0]) > 1e-3 * ev[:, 1]
    dots = np.abs(np.sum(n_gpu[ok].astype(np.float64) * n_ref[ok], axis=1))
    assert np.median(1 - dots) < 1e-8 and np.mean(dots > 1 - 1e-4) > 0.99


def test_knn_batch_equals_one_grid_calls(o3g):
    pts = clouds()
    g = synth.rng(710)
    grids = [o3g.build_grid(cuda(p), 0.05) for p in pts]
    qs = [cuda((p[g.integers(0, len(p), min(len(p), 4000))] + g.normal(0, 0.01, (min(len(p), 4000), 3))).astype(
        np.float32)) if len(p) else cuda(np.zeros((0, 3), np.float32)) for p in pts]
    res = o3g.knn_hybrid_batch(grids, qs, 0.05, 16)
    for grid, q, (idx, d2, cnt) in zip(grids, qs, res):
        i2, dd2, c2 = o3g.knn_hybrid(grid, q, 0.05, 16)
        assert np.array_equal(idx.cpu().numpy(), i2.cpu().numpy())
        assert np.array_equal(d2.cpu().numpy(), dd2.cpu().numpy())
        assert np.array_equal(cnt.cpu().numpy(), c2.cpu().numpy())
    # one set against the oracle's brute-force hybrid search
    k = 4
    i_ref, d_ref, c_ref = oracle.knn_hybrid(pts[k], qs[k].cpu().numpy(), 0.05, 16)
    idx, d2, cnt = res[k]
    assert np.array_equal(cnt.cpu().numpy(), c_ref)
    m = np.arange(16)[None, :] < c_ref[:, None]
    assert np.array_equal(idx.cpu().numpy()[m], i_ref[m]) and np.array_equal(d2.cpu().numpy()[m], d_ref[m])


def test_batch_argument_errors(o3g):
    grid = o3g.build_grid(cuda(np.zeros((5, 3), np.float32)), 0.1)
    with pytest.raises(o3g.O3GError):
        o3g.estimate_normals_batch([grid], -1.0, 30)
    with pytest.raises(o3g.O3GError):
        o3g.estimate_normals_batch([grid], 0.1, 0)
    o3g.estimate_normals_batch([], 0.1, 30)
