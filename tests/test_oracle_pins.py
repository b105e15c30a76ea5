"""Pins of the CPU oracle against what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: brute force
in numpy, finite differences, scipy/numpy library routines, closed forms and
invariants.  The cited passages are those of the Open3D paper (arXiv 1801.09847).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree
from scipy.spatial.transform import Rotation

from paper_1801_09847_gb300 import synth
from tests import _independent as ind

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ a3: transform


def test_transform_identity_is_exact(ora):
    g = synth.rng(10)
    s = g.uniform(-3, 3, (500, 3)).astype(np.float32)
    assert np.array_equal(ora.transform(s, np.eye(4)), s)


def test_transform_within_fp32_rounding_of_fp64(ora):
    """p = R s + t evaluated in FP32 stays within a few ulps of the exact FP64 value."""
    g = synth.rng(11)
    s = g.uniform(-3, 3, (2000, 3)).astype(np.float32)
    T = synth.perturbation(g, 40.0, 0.7)
    p = ora.transform(s, T).astype(np.float64)
    exact = synth.apply_T(T, s.astype(np.float64))
    scale = np.abs(s.astype(np.float64)) @ np.abs(T[:3, :3]).T + np.abs(T[:3, 3])
    assert np.all(np.abs(p - exact) <= 8 * 2.0**-24 * scale)


# ------------------------------------------------------------------ a4: NN


def test_nn_golden_tiny(ora):
    gd = _golden("nn_tiny.json")
    corr, d2 = ora.nn(np.array(gd["queries"], np.float32), np.array(gd["targets"], np.float32), gd["r_max"])
    assert corr.tolist() == gd["corr"]
    assert np.array_equal(d2, np.array(gd["d2"], np.float32))


@pytest.mark.parametrize("ns,nt,r", [(1, 1, 0.3), (257, 1000, 0.2), (1500, 700, 0.5), (64, 2000, 0.05)])
def test_nn_matches_numpy_bruteforce_bitexact(ora, ns, nt, r):
    g = synth.rng(100 + ns)
    tgt = g.uniform(-1, 1, (nt, 3)).astype(np.float32)
    # include duplicates of targets (exact ties) and points far away
    p = g.uniform(-1.2, 1.2, (ns, 3)).astype(np.float32)
    p[: ns // 4] = tgt[g.integers(0, nt, ns // 4)]
    dup = tgt.copy()
    tgt2 = np.vstack([tgt, dup[: nt // 3]])  # later duplicates must lose ties
    c1, d1 = ora.nn(p, tgt2, r, threads=3)
    c2, d2 = ind.nn_bruteforce_f32(p, tgt2, r)
    assert np.array_equal(c1, c2)
    assert np.array_equal(d1, d2)
    assert np.all(c1[: ns // 4] < nt)  # duplicates never win over the lower index


def test_nn_agrees_with_kdtree_where_unambiguous(ora):
    """scipy's kd-tree (FP64 distances) gives the same neighbour wherever the FP64 gap is not tiny."""
    g = synth.rng(12)
    tgt = g.uniform(-1, 1, (3000, 3)).astype(np.float32)
    p = g.uniform(-1, 1, (3000, 3)).astype(np.float32)
    r = 0.15
    corr, d2 = ora.nn(p, tgt, r)
    tree = cKDTree(tgt.astype(np.float64))
    dist, idx = tree.query(p.astype(np.float64), k=2)
    within = dist[:, 0] <= r * (1 - 1e-5)
    clear = (dist[:, 1] - dist[:, 0] > 1e-5) & within
    assert np.array_equal(corr[clear], idx[clear, 0])
    outside = dist[:, 0] > r * (1 + 1e-5)
    assert np.all(corr[outside] == -1)
    assert np.allclose(np.sqrt(d2[clear]), dist[clear, 0], rtol=1e-6, atol=1e-7)


def test_nn_radius_boundary_inclusive(ora):
    r = np.float32(0.05)
    tgt = np.array([[r, 0, 0], [0, np.nextafter(r, np.float32(1)), 0]], np.float32)
    p = np.zeros((1, 3), np.float32)
    corr, d2 = ora.nn(p, tgt, float(r))
    assert corr[0] == 0 and d2[0] == r * r
    corr, _ = ora.nn(p, tgt[1:], float(r))
    d_out = np.float32(tgt[1, 1]) * np.float32(tgt[1, 1])
    assert (corr[0] == -1) == (d_out > r * r)


def test_nn_empty_target(ora):
    p = np.zeros((5, 3), np.float32)
    corr, _ = ora.nn(p, np.zeros((0, 3), np.float32), 1.0)
    assert np.all(corr == -1)


# ------------------------------- a4 at scale: the exact grid search of the oracle


@pytest.mark.parametrize("ns,nt,r,span", [(3000, 3000, 0.05, 1.0), (2000, 5000, 0.2, 1.0), (500, 400, 1.5, 1.0),
                                          (4000, 4000, 0.003, 0.1)])
def test_grid_nn_equals_bruteforce_bitexact(ora, ns, nt, r, span):
    """The grid search is an acceleration of the scan: identical indices and d2 (ties, far points included)."""
    g = synth.rng(700 + ns + nt)
    tgt = g.uniform(-span, span, (nt, 3)).astype(np.float32)
    tgt = np.vstack([tgt, tgt[: nt // 5]])  # exact duplicates: the lower index must win
    p = g.uniform(-1.2 * span, 1.2 * span, (ns, 3)).astype(np.float32)
    p[: ns // 3] = tgt[g.integers(0, nt, ns // 3)] + g.normal(0, r / 3, (ns // 3, 3)).astype(np.float32)
    c1, d1 = ora.nn(p, tgt, r, threads=4)
    c2, d2 = ora.nn(p, tgt, r, threads=3, method="grid")
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)
    assert 0 < np.count_nonzero(c1 >= 0) < ns or r >= 1.0


def test_grid_nn_on_a_lattice_at_the_radius(ora):
    """Targets on a lattice of spacing exactly r: every lattice neighbour sits at d2 == r^2 (inclusive) and the
    queries sit on the lattice, on cell faces and in between, so a missing cell or a strict bound shows."""
    r = 0.25
    ax = np.arange(-4, 5, dtype=np.float32) * np.float32(r)
    tgt = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    g = synth.rng(71)
    tgt = tgt[g.permutation(len(tgt))]
    q = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3) + np.float32(r / 2)
    h = np.float32(1.01 * r)
    faces = (np.arange(-3, 4, dtype=np.float32) * h)
    qf = np.stack(np.meshgrid(faces, faces, faces, indexing="ij"), -1).reshape(-1, 3)
    p = np.vstack([tgt + np.array([r, 0, 0], np.float32), q, qf]).astype(np.float32)
    c1, d1 = ora.nn(p, tgt, r)
    c2, d2 = ora.nn(p, tgt, r, method="grid")
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)
    # a query exactly r from its nearest target (the target shifted by r) matches at d2 == r^2 or closer
    assert np.all(c1[: len(tgt)] >= 0)


def test_grid_nn_partners_at_the_radius_anywhere_in_a_cell(ora):
    """Isolated queries at random offsets, each with one partner about r away along a random axis: the partner
    falls in the neighbouring cell or further whenever the cell is narrower than r, so a cell below r shows."""
    r = 0.05
    g = synth.rng(73)
    n = 20000
    base = np.stack(np.meshgrid(*(np.arange(28),) * 3, indexing="ij"), -1).reshape(-1, 3)[:n] * (10 * r)
    p = (base + g.uniform(0, 3 * r, (n, 3))).astype(np.float32)
    e = np.zeros((n, 3), np.float32)
    e[np.arange(n), g.integers(0, 3, n)] = g.choice([-1.0, 1.0], n) * np.float32(r)
    tgt = (p + e).astype(np.float32)
    c1, d1 = ora.nn(p, tgt, r)
    c2, d2 = ora.nn(p, tgt, r, method="grid")
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)
    assert np.count_nonzero(c1 >= 0) > n // 4


def test_grid_nn_nonfinite_and_far(ora):
    tgt = np.array([[0, 0, 0], [np.nan, 0, 0], [np.inf, 0, 0], [1e30, 1e30, 1e30], [0.01, 0, 0]], np.float32)
    p = np.array([[0.004, 0, 0], [np.nan, 0, 0], [np.inf, 0, 0], [1e30, 1e30, 1e30], [-1e30, 0, 0]], np.float32)
    c1, d1 = ora.nn(p, tgt, 0.05)
    c2, d2 = ora.nn(p, tgt, 0.05, method="grid")
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)
    assert c1.tolist() == [0, -1, -1, 3, -1]


def test_grid_nn_large_offsets(ora):
    """Clouds far from the origin (coarse FP32 spacing) give the same map."""
    g = synth.rng(72)
    tgt = (g.uniform(-1, 1, (3000, 3)) + 1000.0).astype(np.float32)
    p = (tgt[g.integers(0, 3000, 2000)] + g.normal(0, 0.01, (2000, 3))).astype(np.float32)
    c1, d1 = ora.nn(p, tgt, 0.02)
    c2, d2 = ora.nn(p, tgt, 0.02, method="grid")
    assert np.array_equal(c1, c2) and np.array_equal(d1, d2)


def test_icp_with_grid_search_equals_scan(ora):
    """Same correspondences every iteration, so the whole registration is bit-identical."""
    pr = synth.sphere_plane_pair()
    a = ora.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter)
    b = ora.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter, nn_method="grid")
    assert a["status"] == b["status"] and a["iters"] == b["iters"]
    assert np.array_equal(a["T"], b["T"]) and a["fitness"] == b["fitness"] and a["rmse"] == b["rmse"]


# --------------------------------------------------- a5: residual, Jacobian


def test_jacobian_matches_finite_differences(ora):
    """J = [p x n ; n] is the derivative of r(xi) = (exp(xi) p - q) . n at xi = 0 (Eq. 2's J_r)."""
    g = synth.rng(13)
    for _ in range(20):
        p = g.uniform(-2, 2, 3).astype(np.float32)
        q = (p + g.normal(0, 0.05, 3)).astype(np.float32)
        n = synth.random_unit(g).astype(np.float32)
        J, r = ora.residual_jacobian(p, q, n)
        Jfd = ind.fd_jacobian(p[None], q[None], n[None])[0]
        assert np.allclose(J, Jfd, rtol=1e-6, atol=1e-8)
        assert r == pytest.approx(float(np.dot(p.astype(np.float64) - q, n.astype(np.float64))), abs=1e-15)


def _random_corr_problem(g, n=400):
    tgt = g.uniform(-1, 1, (n, 3)).astype(np.float32)
    nrm = np.array([synth.random_unit(g) for _ in range(n)], np.float32)
    p = (tgt + g.normal(0, 0.02, tgt.shape)).astype(np.float32)
    corr = np.arange(n, dtype=np.int32)
    corr[::7] = -1
    d2 = np.sum((p - tgt) ** 2, axis=1).astype(np.float32)
    return p, tgt, nrm, corr, d2


def test_normal_equations_equal_gauss_newton_of_fd_jacobian(ora):
    """A = J^T J and b = J^T r with J from finite differences of the residuals (Eq. 1-2)."""
    g = synth.rng(14)
    p, tgt, nrm, corr, d2 = _random_corr_problem(g)
    A, b, sr2, sd2, cnt = ora.normal_equations(p, tgt, nrm, corr, d2)
    m = corr >= 0
    Jfd = ind.fd_jacobian(p[m], tgt[corr[m]], nrm[corr[m]])
    r = ind.residuals(np.zeros(6), p[m], tgt[corr[m]], nrm[corr[m]])
    assert cnt == m.sum()
    assert np.allclose(A, Jfd.T @ Jfd, rtol=1e-6, atol=1e-9)
    assert np.allclose(b, Jfd.T @ r, rtol=1e-6, atol=1e-10)
    assert sr2 == pytest.approx(float(r @ r), rel=1e-12)
    assert sd2 == pytest.approx(float(np.sum(d2[m].astype(np.float64))), rel=1e-12)


def test_normal_equations_symmetric_psd_and_sign_invariant(ora):
    g = synth.rng(15)
    p, tgt, nrm, corr, d2 = _random_corr_problem(g)
    A, b, *_ = ora.normal_equations(p, tgt, nrm, corr, d2)
    assert np.array_equal(A, A.T)
    ev = np.linalg.eigvalsh(A)
    assert ev.min() >= -1e-12 * ev.max()
    flip = nrm.copy()
    flip[::3] *= -1
    A2, b2, *_ = ora.normal_equations(p, tgt, flip, corr, d2)
    assert np.array_equal(A, A2) and np.array_equal(b, b2)


def test_normal_equations_identity_gives_zero_gradient(ora):
    g = synth.rng(16)
    s = g.uniform(-1, 1, (300, 3)).astype(np.float32)
    nrm = np.array([synth.random_unit(g) for _ in range(300)], np.float32)
    p = ora.transform(s, np.eye(4))
    corr, d2 = ora.nn(p, s, 0.01)
    assert np.array_equal(corr, np.arange(300))
    A, b, sr2, sd2, cnt = ora.normal_equations(p, s, nrm, corr, d2)
    assert np.all(b == 0.0) and sr2 == 0.0 and sd2 == 0.0 and cnt == 300


def test_plane_gives_rank_three(ora):
    g = synth.rng(17)
    tgt = np.column_stack([g.uniform(-1, 1, 500), g.uniform(-1, 1, 500), np.zeros(500)]).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (500, 1))
    p = (tgt + np.array([0, 0, 0.01], np.float32)).astype(np.float32)
    corr = np.arange(500, dtype=np.int32)
    A, b, *_ = ora.normal_equations(p, tgt, nrm, corr, np.zeros(500, np.float32))
    for k in (2, 3, 4):  # gamma, t_x, t_y
        assert np.all(A[k] == 0) and np.all(A[:, k] == 0) and b[k] == 0
    assert np.linalg.matrix_rank(A) == 3


# -------------------------------------------------------------- a6: solve


def test_ldlt_matches_numpy_solve_on_spd(ora):
    g = synth.rng(18)
    for _ in range(50):
        M = g.standard_normal((6, 6))
        A = M @ M.T + 0.1 * np.eye(6)
        b = g.standard_normal(6)
        xi, nf = ora.ldlt_solve(A, b)
        assert nf == 0
        ref = np.linalg.solve(A, -b)
        assert np.linalg.norm(xi - ref) <= 1e-12 * np.linalg.cond(A) * np.linalg.norm(ref)


def test_ldlt_frozen_pivot_solves_reduced_system(ora):
    g = synth.rng(19)
    M = g.standard_normal((6, 6))
    A = M @ M.T + np.eye(6)
    A[[1, 4], :] = 0
    A[:, [1, 4]] = 0
    b = g.standard_normal(6)
    b[[1, 4]] = 0
    xi, nf = ora.ldlt_solve(A, b)
    assert nf == 2 and xi[1] == 0 and xi[4] == 0
    keep = [0, 2, 3, 5]
    ref = np.linalg.solve(A[np.ix_(keep, keep)], -b[keep])
    assert np.allclose(xi[keep], ref, rtol=1e-12, atol=1e-14)


def test_ldlt_all_zero_freezes_everything(ora):
    xi, nf = ora.ldlt_solve(np.zeros((6, 6)), np.ones(6))
    assert nf == 6 and np.all(xi == 0)


def test_delta_T_is_intrinsic_zyx_euler(ora):
    """dR = Rz(gamma) Ry(beta) Rx(alpha): scipy's intrinsic 'ZYX' with angles (gamma, beta, alpha)."""
    g = synth.rng(20)
    for _ in range(20):
        xi = g.uniform(-0.5, 0.5, 6)
        dT = ora.delta_T(xi)
        R = Rotation.from_euler("ZYX", [xi[2], xi[1], xi[0]]).as_matrix()
        assert np.allclose(dT[:3, :3], R, atol=1e-15)
        assert np.array_equal(dT[:3, 3], xi[3:]) and np.array_equal(dT[3], [0, 0, 0, 1])


def test_one_gauss_newton_step_matches_lstsq(ora):
    """The step of Eq. 2 is the least-squares solution of J xi = -r with J from finite differences."""
    g = synth.rng(21)
    p, tgt, nrm, corr, d2 = _random_corr_problem(g, 300)
    A, b, *_ = ora.normal_equations(p, tgt, nrm, corr, d2)
    xi, nf = ora.ldlt_solve(A, b)
    m = corr >= 0
    Jfd = ind.fd_jacobian(p[m], tgt[corr[m]], nrm[corr[m]])
    r = ind.residuals(np.zeros(6), p[m], tgt[corr[m]], nrm[corr[m]])
    ref = np.linalg.lstsq(Jfd, -r, rcond=None)[0]
    assert nf == 0
    assert np.allclose(xi, ref, rtol=1e-5, atol=1e-9)


def test_planar_closed_form_golden(ora):
    """Golden closed-form step on a planar scene (Eq. 2); derivation in tests/golden/planar_step.json."""
    gd = _golden("planar_step.json")
    xs, ys = np.meshgrid(np.linspace(-1, 1, 21), np.linspace(-1, 1, 21))
    tgt = np.column_stack([xs.ravel(), ys.ravel(), np.zeros(xs.size)]).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (len(tgt), 1))
    for case in gd["cases"]:
        a, b_, c = case["a"], case["b"], case["c"]
        src = np.column_stack([xs.ravel(), ys.ravel(), a * xs.ravel() + b_ * ys.ravel() + c]).astype(np.float32)
        p = ora.transform(src, np.eye(4))
        corr = np.arange(len(tgt), dtype=np.int32)  # the vertical neighbour is the correspondence
        d2 = np.sum((p - tgt) ** 2, axis=1).astype(np.float32)
        A, b, *_ = ora.normal_equations(p, tgt, nrm, corr, d2)
        xi, nf = ora.ldlt_solve(A, b)
        assert nf == 3
        assert np.allclose(xi, case["xi"], atol=2e-7), (xi, case["xi"])


# --------------------------------------------------------- whole ICP loop


def _corner_scene(g, spacing=0.02):
    """Three orthogonal 1 x 1 planes (a room corner) plus a sphere: all six DOF observable; analytic normals."""
    u = np.arange(0.0, 1.0, spacing)
    a, b = np.meshgrid(u, u)
    a, b = a.ravel(), b.ravel()
    z0 = np.zeros_like(a)
    P = [np.column_stack([a, b, z0]), np.column_stack([a, z0, b]), np.column_stack([z0, a, b])]
    N = [np.tile([0, 0, 1.0], (len(a), 1)), np.tile([0, 1.0, 0], (len(a), 1)), np.tile([1.0, 0, 0], (len(a), 1))]
    v = g.standard_normal((1500, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    P.append(0.2 * v + np.array([0.5, 0.5, 0.5]))
    N.append(v)
    return np.vstack(P), np.vstack(N)


def test_icp_recovers_known_transform_noise_free(ora):
    """Noise-free source = T_gt^-1 target: ICP returns T_gt (limited by FP32 input rounding), fitness 1."""
    g = synth.rng(22)
    tgt, nrm = _corner_scene(g)
    T_gt = synth.perturbation(g, 2.0, 0.02)
    src = synth.apply_T(synth.inv_T(T_gt), tgt).astype(np.float32)
    res = ora.icp_point_to_plane(src, tgt.astype(np.float32), nrm.astype(np.float32), np.eye(4), 0.05, 30)
    ang, dt = synth.pose_error(res["T"], T_gt)
    assert ang < 1e-6 and dt < 1e-6, (ang, dt)
    assert res["fitness"] == 1.0 and res["rmse"] < 1e-6 and res["status"] == 0


def test_icp_equivariance(ora):
    """Moving both clouds by G turns the result T into G T G^-1."""
    g = synth.rng(23)
    tgt, nrm = _corner_scene(g, spacing=0.03)
    T_gt = synth.perturbation(g, 2.0, 0.02)
    src = synth.apply_T(synth.inv_T(T_gt), tgt) + g.normal(0, 0.001, tgt.shape)
    G = synth.perturbation(g, 30.0, 0.5)
    r1 = ora.icp_point_to_plane(src.astype(np.float32), tgt.astype(np.float32), nrm.astype(np.float32),
                                np.eye(4), 0.05, 20)
    tgt_g = synth.apply_T(G, tgt)
    nrm_g = nrm @ G[:3, :3].T
    r2 = ora.icp_point_to_plane(synth.apply_T(G, src).astype(np.float32), tgt_g.astype(np.float32),
                                nrm_g.astype(np.float32), np.eye(4), 0.05, 20)
    ang, dt = synth.pose_error(r2["T"], G @ r1["T"] @ synth.inv_T(G))
    assert ang < 1e-5 and dt < 1e-5, (ang, dt)


def test_icp_few_correspondences_status(ora):
    g = synth.rng(24)
    tgt = g.uniform(-1, 1, (100, 3)).astype(np.float32)
    src = (tgt + 10.0).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (100, 1))
    T0 = np.eye(4)
    res = ora.icp_point_to_plane(src, tgt, nrm, T0, 0.1, 10)
    assert res["status"] == ora.WARN_FEW_CORR and res["iters"] == 0
    assert np.array_equal(res["T"], T0) and res["fitness"] == 0.0 and res["rmse"] == 0.0


def test_icp_planar_scene_is_degenerate(ora):
    g = synth.rng(25)
    tgt = np.column_stack([g.uniform(-1, 1, 800), g.uniform(-1, 1, 800), np.zeros(800)]).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (800, 1))
    src = (tgt + np.array([0, 0, 0.01], np.float32)).astype(np.float32)
    res = ora.icp_point_to_plane(src, tgt, nrm, np.eye(4), 0.1, 5)
    assert res["status"] == ora.WARN_DEGENERATE
    assert abs(res["T"][2, 3] + 0.01) < 1e-6  # t_z recovered; the in-plane DOF stay frozen


def test_icp_sphere_plane_config_runs(ora):
    """The 4,096-point sphere-plus-plane pair: all source points find partners and the rmse is near the noise."""
    pr = synth.sphere_plane_pair()
    res = ora.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter)
    assert res["iters"] == 30 and res["fitness"] > 0.99
    ang, dt = synth.pose_error(res["T"], pr.T_gt)
    assert dt < 2e-3  # rotation about z is unobservable for this scene (see the scene notes)


def test_max_iter_zero_is_evaluation_only(ora):
    pr = synth.sphere_plane_pair(n=500)
    res = ora.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), 0.05, 0)
    assert res["iters"] == 0 and np.array_equal(res["T"], np.eye(4))
    p = ora.transform(pr.src, np.eye(4))
    corr, d2 = ind.nn_bruteforce_f32(p, pr.tgt, 0.05)
    m = corr >= 0
    assert res["fitness"] == m.sum() / len(p)
    assert res["rmse"] == pytest.approx(math.sqrt(np.sum(d2[m].astype(np.float64)) / m.sum()), rel=1e-12)


# ------------------------------------------------------------- a2: normals


def test_knn_matches_numpy_bruteforce(ora):
    g = synth.rng(26)
    pts = g.uniform(-0.3, 0.3, (1200, 3)).astype(np.float32)
    pts[100:120] = pts[0]  # exact ties
    q = pts[::5]
    for radius, k in [(0.1, 30), (0.05, 7), (0.5, 64)]:
        idx, dd, cnt = ora.knn_hybrid(pts, q, radius, k)
        for i in range(len(q)):
            ri, rd = ind.knn_bruteforce_f32(pts, q[i], radius, k)
            assert cnt[i] == len(ri)
            assert np.array_equal(idx[i, : cnt[i]], ri) and np.array_equal(dd[i, : cnt[i]], rd)
            assert np.all(idx[i, cnt[i]:] == -1)


def test_knn_radius_boundary_and_ties(ora):
    """Hybrid kNN on an exact binary lattice (spacing 0.25, shuffled, with duplicates at higher indices):
    the radius is inclusive, equal distances go to the lower index, and the count within radius 0.5 of a
    lattice point is the closed form: integer triples with i^2 + j^2 + k^2 <= 4 number 1 + 6 + 12 + 8 + 6 = 33."""
    g = synth.rng(31)
    ax = np.arange(-4, 5) * 0.25
    lat = np.stack(np.meshgrid(ax, ax, ax, indexing="ij"), -1).reshape(-1, 3)
    lat = lat[g.permutation(len(lat))]
    pts = np.vstack([lat, lat[:40]]).astype(np.float32)  # 40 exact copies after all originals
    q = np.array([[0, 0, 0], [0.125, 0.125, 0.125], [0.25, -0.5, 0.75]], np.float32)
    for radius, k in [(0.5, 64), (0.5, 7), (0.25, 27), (0.5, 1)]:
        idx, dd, cnt = ora.knn_hybrid(pts, q, radius, k)
        for i in range(len(q)):
            ri, rd = ind.knn_bruteforce_f32(pts, q[i], radius, k)
            assert cnt[i] == len(ri)
            assert np.array_equal(idx[i, : cnt[i]], ri) and np.array_equal(dd[i, : cnt[i]], rd)
        # at the origin: the 33 lattice points within 0.5, plus whichever of them were copied
        near = np.flatnonzero(np.sum(lat.astype(np.float64) ** 2, 1) <= radius * radius)
        copies = np.count_nonzero(np.isin(np.arange(40), near))
        assert cnt[0] == min(k, len(near) + copies)
        if radius == 0.5:
            assert len(near) == 33
        # ties go to the lower index: among equal d2, indices ascend
        for a in range(cnt[0] - 1):
            assert dd[0, a] < dd[0, a + 1] or idx[0, a] < idx[0, a + 1]


def test_jacobi_matches_numpy_eigh(ora):
    g = synth.rng(27)
    for _ in range(200):
        M = g.standard_normal((3, 3))
        C = M @ M.T * g.uniform(1e-6, 1.0)
        ev, V = ora.jacobi_eig3(C)
        ref = np.linalg.eigvalsh(C)
        assert np.allclose(np.sort(ev), ref, rtol=1e-12, atol=1e-14 * ref.max())
        assert np.allclose(C @ V, V * ev[None, :], atol=1e-12 * ref.max())
        assert np.allclose(V.T @ V, np.eye(3), atol=1e-13)


def test_normals_on_plane_are_exact(ora):
    g = synth.rng(28)
    pts = np.column_stack([g.uniform(-1, 1, 2000), g.uniform(-1, 1, 2000), np.full(2000, 0.25)]).astype(np.float32)
    nrm = ora.estimate_normals(pts, 0.1, 30, viewpoint=(0.0, 0.0, 5.0))
    assert np.array_equal(nrm, np.tile(np.array([0, 0, 1], np.float32), (2000, 1)))
    nrm = ora.estimate_normals(pts, 0.1, 30, viewpoint=(0.0, 0.0, -5.0))
    assert np.array_equal(nrm, np.tile(np.array([0, 0, -1], np.float32), (2000, 1)))


def test_normals_on_sphere_are_radial_and_oriented(ora):
    g = synth.rng(29)
    v = g.standard_normal((20000, 3))  # ~50 points within 0.1, so the 30 nearest span a small cap
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pts = v.astype(np.float32)
    nrm = ora.estimate_normals(pts, 0.1, 30, viewpoint=(0.0, 0.0, 0.0))
    n64 = nrm.astype(np.float64)
    ang = np.arctan2(np.linalg.norm(np.cross(n64, v), axis=1), np.abs(np.sum(n64 * v, axis=1)))
    # a plane fitted to a cap of angular radius 0.1 tilts by at most about half of it when the
    # neighbours are lopsided; a wrong eigenvector would be off by ~90 degrees
    assert np.all(ang < 0.05) and np.median(ang) < 1e-2
    assert np.all(np.sum(nrm * (0 - pts), axis=1) >= 0)  # facing the centre viewpoint


def test_normals_few_neighbours_default(ora):
    pts = np.array([[0, 0, 0], [0.01, 0, 0], [5, 5, 5]], np.float32)
    nrm = ora.estimate_normals(pts, 0.05, 30)
    assert np.array_equal(nrm, np.tile(np.array([0, 0, 1], np.float32), (3, 1)))


def test_normals_match_eigh_of_neighbour_covariance(ora):
    """The normal is numpy.linalg.eigh's smallest eigenvector of the neighbourhood covariance."""
    g = synth.rng(30)
    pts = (g.uniform(-0.2, 0.2, (800, 3)) * np.array([1, 1, 0.2])).astype(np.float32)
    radius, k = 0.1, 30
    nrm, ev = ora.estimate_normals(pts, radius, k, viewpoint=(0.0, 0.0, 1.0), return_evals=True)
    for i in range(0, 800, 13):
        idx, _ = ind.knn_bruteforce_f32(pts, pts[i], radius, k)
        X = pts[idx].astype(np.float64)
        C = np.cov(X.T, bias=True)
        w, V = np.linalg.eigh(C)
        assert np.allclose(ev[i], w, rtol=1e-9, atol=1e-15)
        if w[1] - w[0] > 1e-3 * w[2]:
            cosang = abs(float(np.dot(nrm[i].astype(np.float64), V[:, 0])))
            assert cosang > 1 - 2e-7  # FP32 storage of a unit vector


# ------------------------------------------ point-to-point ICP (Horn's closed form)


def _kabsch_svd(p, q):
    """Independent statement of the least-squares rigid motion: SVD of the centred cross-covariance
    (Kabsch / Umeyama without scale, with the determinant correction that keeps R a rotation)."""
    p = p.astype(np.float64)
    q = q.astype(np.float64)
    mp, mq = p.mean(0), q.mean(0)
    H = (p - mp).T @ (q - mq)
    U, _, Vt = np.linalg.svd(H)
    d = np.sign(np.linalg.det(Vt.T @ U.T))
    R = Vt.T @ np.diag([1.0, 1.0, d]) @ U.T
    return synth.make_T(R, mq - R @ mp)


def test_jacobi4_matches_numpy_eigh(ora):
    g = synth.rng(80)
    for _ in range(20):
        M = g.normal(size=(4, 4))
        C = M + M.T
        ev, V = ora.jacobi_eig4(C)
        ref = np.linalg.eigvalsh(C)
        assert np.allclose(np.sort(ev), ref, rtol=0, atol=1e-12 * np.abs(ref).max())
        assert np.allclose(C @ V, V * ev, atol=1e-11 * np.abs(ref).max())
        assert np.allclose(V.T @ V, np.eye(4), atol=1e-13)


@pytest.mark.parametrize("noise,deg,trans", [(0.0, 30.0, 0.5), (0.01, 10.0, 0.1), (0.05, 170.0, 2.0)])
def test_rigid_align_matches_svd_kabsch(ora, noise, deg, trans):
    g = synth.rng(81 + int(deg))
    p = g.normal(0, 1, (500, 3)).astype(np.float32)
    T = synth.perturbation(g, deg, trans)
    q = (synth.apply_T(T, p) + g.normal(0, noise, p.shape)).astype(np.float32)
    # a partial correspondence map: some points unmatched, targets in shuffled order
    perm = g.permutation(500)
    tgt = q[perm]
    corr = np.argsort(perm).astype(np.int32)
    corr[g.random(500) < 0.2] = -1
    dT, deg_flag, ang, cnt = ora.rigid_align(p, tgt, corr)
    m = corr >= 0
    ref = _kabsch_svd(p[m], tgt[corr[m]])
    assert not deg_flag and cnt == m.sum()
    assert np.allclose(dT, ref, atol=1e-10)
    R = dT[:3, :3]
    assert np.allclose(R @ R.T, np.eye(3), atol=1e-13) and np.linalg.det(R) == pytest.approx(1.0, abs=1e-13)
    assert ang == pytest.approx(np.arccos(np.clip((np.trace(R) - 1) / 2, -1, 1)), abs=1e-7)
    if noise == 0.0:
        a, t = synth.pose_error(dT, T)
        assert a < 1e-6 and t < 1e-6


def test_rigid_align_best_rotation_for_a_mirrored_cloud(ora):
    """A reflected target: the answer is the best proper rotation, as the determinant-corrected SVD gives."""
    g = synth.rng(84)
    p = (g.normal(0, 1, (300, 3)) * [3.0, 2.0, 1.0]).astype(np.float32)
    q = (p * np.float32([1, 1, -1])).astype(np.float32)
    dT, deg_flag, _, _ = ora.rigid_align(p, q, np.arange(300, dtype=np.int32))
    assert not deg_flag
    assert np.allclose(dT, _kabsch_svd(p, q), atol=1e-10)


def test_rigid_align_collinear_is_degenerate(ora):
    t = np.linspace(-1, 1, 50)
    p = np.stack([t, 2 * t, -t], 1).astype(np.float32)
    q = (p + np.float32([0.1, 0.2, 0.3])).astype(np.float32)
    dT, deg_flag, ang, _ = ora.rigid_align(p, q, np.arange(50, dtype=np.int32))
    assert deg_flag and ang == 0.0
    assert np.array_equal(dT[:3, :3], np.eye(3))
    assert np.allclose(dT[:3, 3], q.astype(np.float64).mean(0) - p.astype(np.float64).mean(0), atol=1e-15)


def test_icp_point_to_point_recovers_noise_free(ora):
    pr = synth.sphere_plane_pair(noise=0.0, deg=3.0, trans=0.02)
    res = ora.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 200, eps=1e-9)
    a, t = synth.pose_error(res["T"], pr.T_gt)
    assert a < 1e-5 and t < 1e-5, (a, t, res)
    assert res["fitness"] == 1.0 and res["rmse"] < 1e-5


def test_icp_point_to_point_equivariance(ora):
    """Moving both clouds by G conjugates the result (within FP32 input rounding)."""
    pr = synth.sphere_plane_pair(n=2000, noise=0.002, deg=3.0, trans=0.02)
    a = ora.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 30)
    G = synth.make_T(synth.axis_angle_matrix([0.3, -1.0, 0.5], 0.7), [0.5, -0.2, 0.1])
    b = ora.icp_point_to_point(synth.apply_T(G, pr.src).astype(np.float32),
                               synth.apply_T(G, pr.tgt).astype(np.float32), np.eye(4), 0.05, 30)
    ang, dt = synth.pose_error(b["T"], G @ a["T"] @ np.linalg.inv(G))
    assert ang < 1e-4 and dt < 1e-4
    assert abs(a["fitness"] - b["fitness"]) < 0.01


def test_icp_point_to_point_grid_equals_scan_and_statuses(ora):
    pr = synth.sphere_plane_pair(n=3000)
    a = ora.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 20)
    b = ora.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 20, nn_method="grid")
    assert a["status"] == b["status"] == ora.OK and a["iters"] == b["iters"] == 20
    assert np.array_equal(a["T"], b["T"]) and a["rmse"] == b["rmse"]
    far = ora.icp_point_to_point(pr.src + np.float32(10), pr.tgt, np.eye(4), 0.05, 5)
    assert far["status"] == ora.WARN_FEW_CORR and far["iters"] == 0 and far["fitness"] == 0.0
    # eps stops the loop once the update is small
    c = ora.icp_point_to_point(pr.src, pr.tgt, np.eye(4), 0.05, 500, eps=1e-7)
    assert c["iters"] < 500


# ------------------------------------------------------------- voxel downsampling


def _voxel_numpy(p, v):
    """Independent statement: float32 quotients, stable lexicographic order, FP64 sums accumulated in input
    order by bincount."""
    ok = np.all(np.isfinite(p), axis=1)
    p = p[ok]
    k = np.floor(p / np.float32(v)).astype(np.int64)
    uniq, inv = np.unique(k, axis=0, return_inverse=True)  # rows sorted lexicographically, x first
    inv = inv.ravel()
    cnt = np.bincount(inv, minlength=len(uniq))
    c = np.stack([np.bincount(inv, weights=p[:, a].astype(np.float64), minlength=len(uniq)) for a in range(3)], 1)
    return (c / cnt[:, None]).astype(np.float32), cnt.astype(np.int32)


@pytest.mark.parametrize("n,v,span", [(20000, 0.1, 1.0), (5000, 0.013, 0.2), (3000, 5.0, 1.0), (1, 0.1, 1.0)])
def test_voxel_downsample_matches_numpy_bitexact(ora, n, v, span):
    g = synth.rng(90 + n)
    p = g.uniform(-span, span, (n, 3)).astype(np.float32)
    if n > 10:
        p[: n // 10] = (np.round(p[: n // 10] / np.float32(v)) * np.float32(v)).astype(np.float32)  # on voxel faces
        p[n // 10: n // 5] = p[: n // 10]  # duplicates
    c, cnt = ora.voxel_down_sample(p, v)
    c_ref, cnt_ref = _voxel_numpy(p, v)
    assert np.array_equal(cnt, cnt_ref) and np.array_equal(c, c_ref)
    assert cnt.sum() == n


def test_voxel_downsample_properties(ora):
    g = synth.rng(95)
    p = g.normal(0, 1, (5000, 3)).astype(np.float32)
    v = 0.25
    c, cnt = ora.voxel_down_sample(p, v)
    keys = np.floor(c / np.float32(v)).astype(np.int64)
    # the centroid of a voxel's points lies in that voxel, and voxels come in increasing key order
    in_keys = np.unique(np.floor(p / np.float32(v)).astype(np.int64), axis=0)
    assert np.array_equal(keys, in_keys)
    order = np.lexsort(keys.T[::-1])
    assert np.array_equal(order, np.arange(len(c)))  # increasing (ix, iy, iz)
    # one point per voxel: the output is the input point itself
    q = (np.arange(50, dtype=np.float32)[:, None] * np.float32(v) + np.float32(v / 2)) * np.ones((1, 3), np.float32)
    cq, nq = ora.voxel_down_sample(q, v)
    assert np.array_equal(cq, q) and np.all(nq == 1)
    # input order changes at most the last bits of a centroid
    perm = g.permutation(len(p))
    c2, cnt2 = ora.voxel_down_sample(p[perm], v)
    assert np.array_equal(cnt, cnt2) and np.allclose(c, c2, rtol=0, atol=1e-6)


def test_voxel_downsample_edge_cases(ora):
    c, cnt = ora.voxel_down_sample(np.zeros((0, 3), np.float32), 0.1)
    assert len(c) == 0 and len(cnt) == 0
    p = np.array([[0, 0, 0], [np.nan, 0, 0], [0.01, 0.02, 0.03], [np.inf, 1, 1]], np.float32)
    c, cnt = ora.voxel_down_sample(p, 0.1)
    assert cnt.tolist() == [2] and np.array_equal(c[0], np.float32([0.005, 0.01, 0.015]))
    with pytest.raises(ValueError):
        ora.voxel_down_sample(np.array([[1e9, 0, 0]], np.float32), 0.1)
    with pytest.raises(ValueError):
        ora.voxel_down_sample(p, 0.0)


# ----------------------------------------------- hypothesis validation (RANSAC)


def test_evaluate_poses_matches_independent_bruteforce(ora):
    """Counts from an independent numpy float32 brute force; rmse from the same matches summed in FP64."""
    g = synth.rng(120)
    tgt = g.uniform(-1, 1, (1500, 3)).astype(np.float32)
    src = (tgt[g.integers(0, 1500, 800)] + g.normal(0, 0.01, (800, 3))).astype(np.float32)
    poses = [np.eye(4)] + [synth.perturbation(g, d, t) for d, t in ((1.0, 0.01), (5.0, 0.05), (90.0, 1.0))]
    fit, rmse, cnt = ora.evaluate_poses(src, tgt, poses, 0.05)
    for h, T in enumerate(poses):
        p = ora.transform(src, T)
        c, d2 = ind.nn_bruteforce_f32(p, tgt, 0.05)
        m = c >= 0
        assert cnt[h] == m.sum() and fit[h] == m.sum() / len(src)
        ref = np.sqrt(np.sum(d2[m].astype(np.float64)) / m.sum()) if m.any() else 0.0
        assert rmse[h] == pytest.approx(ref, rel=1e-12)
    assert cnt[0] > cnt[3]  # the true pose explains more points than a far-off one
    f2, r2, c2 = ora.evaluate_poses(src, tgt, poses, 0.05, nn_method="grid")
    assert np.array_equal(c2, cnt) and np.array_equal(r2, rmse) and np.array_equal(f2, fit)


def test_evaluate_poses_equals_zero_iteration_icp(ora):
    """Evaluation at a pose is the final-evaluation step of ICP with no update."""
    pr = synth.sphere_plane_pair(n=2000)
    T = synth.perturbation(synth.rng(121), 2.0, 0.02)
    fit, rmse, _ = ora.evaluate_poses(pr.src, pr.tgt, [T], 0.05)
    res = ora.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, T, 0.05, 0)
    assert fit[0] == res["fitness"] and rmse[0] == res["rmse"]
