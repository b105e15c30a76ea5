"""Batched ICP (many pairs per launch) against the single-pair path and the oracle (GPU).

Each pair in a batch must come out bit-identical to the same registration run
alone (same arithmetic, same order), whatever else is in the batch and in
whatever order; a well-conditioned pair must also meet the oracle end to end.
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


def _corner(g, spacing=0.02):
    u = np.arange(0.0, 1.0, spacing)
    a, b = np.meshgrid(u, u)
    a, b = a.ravel(), b.ravel()
    z0 = np.zeros_like(a)
    P = [np.column_stack([a, b, z0]), np.column_stack([a, z0, b]), np.column_stack([z0, a, b])]
    N = [np.tile([0, 0, 1.0], (len(a), 1)), np.tile([0, 1.0, 0], (len(a), 1)), np.tile([1.0, 0, 0], (len(a), 1))]
    return np.vstack(P).astype(np.float32), np.vstack(N).astype(np.float32)


@pytest.fixture(scope="module")
def problems(o3g):
    """A mixed batch: uneven sphere-plane pairs, a corner scene, an empty source, a source far away."""
    probs = []
    for k, n in enumerate([2000, 37, 15000, 4096, 60000]):
        pr = synth.sphere_plane_pair(n=n, seed=500 + k)
        probs.append((pr.tgt, pr.tgt_nrm, pr.src, np.eye(4), pr.max_corr_dist))
    g = synth.rng(9)
    tgt, nrm = _corner(g)
    T_gt = synth.perturbation(g, 2.0, 0.02)
    src = (synth.apply_T(synth.inv_T(T_gt), tgt) + g.normal(0, 0.001, tgt.shape)).astype(np.float32)
    probs.append((tgt, nrm, src, np.eye(4), 0.05))
    probs.append((tgt, nrm, np.zeros((0, 3), np.float32), np.eye(4), 0.05))
    probs.append((tgt, nrm, (tgt[:500] + 20.0).astype(np.float32), np.eye(4), 0.05))
    out = []
    for tgt, nrm, src, T0, r in probs:
        grid = o3g.build_grid(cuda(tgt), r * 1.002)
        grid.set_normals(cuda(nrm))
        out.append((grid, cuda(src), T0, r, src, tgt, nrm))
    return out


def _same(a, b):
    assert a["status"] == b["status"] and a["iters"] == b["iters"]
    assert np.array_equal(a["T"], b["T"])
    assert a["fitness"] == b["fitness"] and a["rmse"] == b["rmse"]


def test_batch_equals_each_pair_alone(o3g, problems):
    alone = [o3g.icp_point_to_plane_grid(g, s, T0, r, 20) for g, s, T0, r, *_ in problems]
    batch = o3g.icp_point_to_plane_batch([p[0] for p in problems], [p[1] for p in problems],
                                         [p[2] for p in problems], [p[3] for p in problems], 20)
    for a, b in zip(alone, batch):
        _same(a, b)
    assert batch[-2]["status"] == o3g.WARN_FEW_CORR and batch[-1]["status"] == o3g.WARN_FEW_CORR


def test_batch_order_and_company_do_not_matter(o3g, problems):
    full = o3g.icp_point_to_plane_batch([p[0] for p in problems], [p[1] for p in problems],
                                        [p[2] for p in problems], [p[3] for p in problems], 15, eps=1e-7)
    perm = synth.rng(3).permutation(len(problems))
    shuffled = o3g.icp_point_to_plane_batch([problems[k][0] for k in perm], [problems[k][1] for k in perm],
                                            [problems[k][2] for k in perm], [problems[k][3] for k in perm], 15,
                                            eps=1e-7)
    for j, k in enumerate(perm):
        _same(full[k], shuffled[j])
    sub = o3g.icp_point_to_plane_batch([problems[1][0], problems[4][0]], [problems[1][1], problems[4][1]],
                                       [problems[1][2], problems[4][2]], [problems[1][3], problems[4][3]], 15,
                                       eps=1e-7)
    _same(full[1], sub[0])
    _same(full[4], sub[1])


def test_batch_pair_matches_oracle(o3g, problems):
    grid, d_src, T0, r, src, tgt, nrm = problems[5]
    res = o3g.icp_point_to_plane_batch([grid, problems[2][0]], [d_src, problems[2][1]], [T0, np.eye(4)], [r, 0.05],
                                       100, eps=1e-7)[0]
    ref = oracle.icp_point_to_plane(src, tgt, nrm, T0, r, 100, eps=1e-7)
    assert res["iters"] == ref["iters"] < 100
    ang, dt = synth.pose_error(res["T"], ref["T"])
    assert ang <= 1e-6 and dt <= 1e-6, (ang, dt)


def test_batch_errors(o3g, problems):
    bare = o3g.build_grid(cuda(problems[0][5]), 0.05)
    with pytest.raises(o3g.O3GError) as e:
        o3g.icp_point_to_plane_batch([problems[0][0], bare], [problems[0][1], problems[0][1]],
                                     [np.eye(4), np.eye(4)], 0.05, 3)
    assert e.value.status == o3g.ERR_ARG
    bad = np.eye(4)
    bad[1, 3] = np.nan
    with pytest.raises(o3g.O3GError) as e:
        o3g.icp_point_to_plane_batch([problems[0][0]], [problems[0][1]], [bad], 0.05, 3)
    assert e.value.status == o3g.ERR_NONFINITE
    nan_src = problems[0][4].copy()
    nan_src[3, 0] = np.nan
    res = o3g.icp_point_to_plane_batch([problems[0][0], problems[2][0]], [cuda(nan_src), problems[2][1]],
                                       [np.eye(4), np.eye(4)], 0.05, 3)
    assert res[0]["status"] == o3g.ERR_NONFINITE and res[1]["status"] >= 0
    assert o3g.icp_point_to_plane_batch([], [], [], 0.05, 3) == []


def test_autotune_picks_a_measured_candidate_and_pins_it(o3g, problems):
    import torch
    from paper_1801_09847_gb300 import autotune
    # problem tuples: (grid, src device, T0, r, src, tgt, nrm); every radius here is 0.05
    assert all(p[3] == 0.05 for p in problems)
    tgts = [cuda(p[5]) for p in problems]
    nrms = [cuda(p[6]) for p in problems]
    srcs = [p[1] for p in problems]
    cls = o3g.size_class(autotune.batch_tiles(srcs))
    try:
        res = autotune.tune_batch(tgts, nrms, srcs, 0.05, iters=2, reps=1, cell_factors=(1.002, 1.5))
        assert set(res["timings_ms"]) == {(cf, f) for cf in (1.002, 1.5) for f in autotune.DEFAULT_FORMS}
        assert res["timings_ms"][(res["cell_factor"], res["form"])] == min(res["timings_ms"].values())
        assert res["size_class"] == cls and o3g.get_tile_config(cls) == res["form"]
        # tuning changes time only: the tuned batch gives the untuned results
        grids = []
        for t, n in zip(tgts, nrms):
            g = o3g.build_grid(t, 0.05 * res["cell_factor"])
            g.set_normals(n)
            grids.append(g)
        tuned = o3g.icp_point_to_plane_batch(grids, srcs, [np.eye(4)] * len(srcs), 0.05, 10)
        o3g.set_tile_config(cls, o3g.TILE_AUTO)
        plain = []
        for t, n in zip(tgts, nrms):
            g = o3g.build_grid(t, 0.05 * 1.002)
            g.set_normals(n)
            plain.append(g)
        ref = o3g.icp_point_to_plane_batch(plain, srcs, [np.eye(4)] * len(srcs), 0.05, 10)
        assert all(np.array_equal(a["T"], b["T"]) for a, b in zip(tuned, ref))
    finally:
        o3g.set_tile_config(cls, o3g.TILE_AUTO)


def test_points_per_thread_alone_batch_and_oracle(o3g, problems):
    """Points per thread (the autotuner's tile-size knob) pinned to 1, 2 and 4 for the pairs' size classes: a
    pair still gives the same result alone and in the batch bit for bit (the setting belongs to the pair's size
    class), the correspondence set at the final pose is the oracle's bit for bit, and every iterate of the
    well-conditioned corner pair is the oracle's Gauss-Newton step from the previous one (1e-7 rad / m)."""
    classes = sorted({o3g.pair_size_class(int(p[1].shape[0])) for p in problems})
    grid, d_src, T0, r, src, tgt, nrm = problems[5]
    try:
        for ppt in (1, 2, 4):
            for c in classes:
                o3g.set_points_per_thread(c, ppt)
                assert o3g.get_points_per_thread(c) == ppt
            alone = [o3g.icp_point_to_plane_grid(g, s, T, rr, 12) for g, s, T, rr, *_ in problems]
            batch = o3g.icp_point_to_plane_batch([p[0] for p in problems], [p[1] for p in problems],
                                                 [p[2] for p in problems], [p[3] for p in problems], 12)
            for a, b in zip(alone, batch):
                _same(a, b)
            res = o3g.icp_point_to_plane_grid(grid, d_src, T0, r, 12, correspondences=True)
            p = oracle.transform(src, res["T"])
            c_ref, d_ref = oracle.nn(p, tgt, r)
            assert np.array_equal(res["corr"].cpu().numpy(), c_ref) and np.array_equal(res["d2"].cpu().numpy(), d_ref)
            T = T0
            for k in range(1, 6):
                Tk = o3g.icp_point_to_plane_grid(grid, d_src, T0, r, k)["T"]
                pk = oracle.transform(src, T)
                corr, d2 = oracle.nn(pk, tgt, r)
                A, b, _, _, _ = oracle.normal_equations(pk, tgt, nrm, corr, d2)
                xi, _ = oracle.ldlt_solve(A, b)
                ang, dt = synth.pose_error(Tk, oracle.delta_T(xi) @ T)
                assert ang <= 1e-7 and dt <= 1e-7, (ppt, k, ang, dt)
                T = Tk
        with pytest.raises(o3g.O3GError):
            o3g.set_points_per_thread(classes[0], 3)
    finally:
        for c in classes:
            o3g.set_points_per_thread(c, 0)
