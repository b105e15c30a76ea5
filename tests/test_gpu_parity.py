"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on seeded inputs.

Bars (Open3D paper, Sec. 3.3 and Sec. 4, Eq. 1-2):
  * correspondences and kNN sets: bit-exact (index and float32 d2);
  * J^T J: ||dA||_F / ||A||_F <= 1e-5;  J^T r: ||db||_inf / ||sum_i |J_i| |r_i|||_inf <= 1e-5;
  * ICP: every GPU iterate T_{k+1} equals the oracle's Gauss-Newton step from the GPU's own T_k within
    1e-7 rad / 1e-7 m ("shadow" check); the final pose within 1e-6 rad and 1e-6 m where the problem is
    well-conditioned and run to convergence, and within max(1e-6, 20 x the oracle's own sensitivity to a
    1e-9 change of the initial pose) where it is not;
  * normals: angle bound scaled by the eigen-gap of the neighbourhood covariance,
    orientation agreeing wherever the normal is not nearly perpendicular to the view ray.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

import oracle
from paper_1801_09847_gb300 import synth

pytestmark = pytest.mark.gpu

POSE_TOL = 1e-6


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


def poses(seed, count=3, deg=4.0, trans=0.04):
    g = synth.rng(seed)
    return [np.eye(4)] + [synth.perturbation(g, deg, trans) for _ in range(count)]


def tie_cloud(g, n, lo=-1.0, hi=1.0, quant=None):
    pts = g.uniform(lo, hi, (n, 3))
    if quant:
        pts = np.round(pts / quant) * quant  # many exactly equal distances
    pts = pts.astype(np.float32)
    pts[n // 2: n // 2 + n // 8] = pts[: n // 8]  # duplicate points: later copies must lose ties
    return pts


# ------------------------------------------------------------ correspondences


# cell factors cover every search variant: window W = 1 (2.0, 1.002), W = 2 (1.0, 0.501),
# W = 3 (0.5, 0.334) and the generic search (0.3)
@pytest.mark.parametrize("ns,nt,r,cell_factor,quant", [
    (1, 1, 0.3, 1.0, None),
    (1000, 3000, 0.1, 1.0, None),
    (2049, 1500, 0.1, 0.5, 0.025),
    (4097, 4096, 0.05, 2.0, None),
    (777, 5001, 0.2, 0.3, 0.05),
    (513, 20000, 0.03, 1.0, None),
    (3001, 6000, 0.08, 1.002, 0.02),
    (2500, 6000, 0.08, 0.501, 0.02),
    (1999, 6000, 0.08, 0.334, 0.02),
])
def test_correspondences_bitexact_random(o3g, ns, nt, r, cell_factor, quant):
    g = synth.rng(1000 + ns)
    tgt = tie_cloud(g, nt, quant=quant)
    src = tie_cloud(g, ns, -1.1, 1.1, quant=quant)
    grid = o3g.build_grid(cuda(tgt), r * cell_factor)
    for T in poses(ns, 2, deg=2.0, trans=0.02):
        corr, d2 = o3g.correspondences(grid, cuda(src), T, r)
        p = oracle.transform(src, T)
        c_ref, d_ref = oracle.nn(p, tgt, r)
        assert np.array_equal(corr.cpu().numpy(), c_ref)
        assert np.array_equal(d2.cpu().numpy(), d_ref)


def test_correspondences_sphere_plane(o3g):
    pr = synth.sphere_plane_pair()
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    for T in poses(7, 4, deg=5.0, trans=0.05) + [pr.T_gt]:
        corr, d2 = o3g.correspondences(grid, cuda(pr.src), T, pr.max_corr_dist)
        c_ref, d_ref = oracle.nn(oracle.transform(pr.src, T), pr.tgt, pr.max_corr_dist)
        assert np.array_equal(corr.cpu().numpy(), c_ref)
        assert np.array_equal(d2.cpu().numpy(), d_ref)


@pytest.fixture(scope="module")
def room():
    return synth.room_frame_pair()


@pytest.mark.parametrize("cell_factor", [1.0, 0.501, 1.002])
def test_correspondences_room_frame_full_size_sampled(o3g, room, cell_factor):
    """The RGB-D-frame pair at full size, in the bench's launch configuration; oracle on a sample of sources."""
    grid = o3g.build_grid(cuda(room.tgt), room.max_corr_dist * cell_factor)
    g = synth.rng(3)
    sample = np.sort(g.choice(len(room.src), 3000, replace=False))
    for T in [np.eye(4), room.T_gt, synth.perturbation(g, 1.0, 0.01) @ room.T_gt]:
        corr, d2 = o3g.correspondences(grid, cuda(room.src), T, room.max_corr_dist)
        c_ref, d_ref = oracle.nn(oracle.transform(room.src[sample], T), room.tgt, room.max_corr_dist)
        assert np.array_equal(corr.cpu().numpy()[sample], c_ref)
        assert np.array_equal(d2.cpu().numpy()[sample], d_ref)


def test_correspondences_edge_cases(o3g):
    g = synth.rng(5)
    tgt = g.uniform(-1, 1, (100, 3)).astype(np.float32)
    src = g.uniform(-1, 1, (50, 3)).astype(np.float32)
    # empty target: no correspondences
    empty = o3g.build_grid(cuda(np.zeros((0, 3), np.float32)), 0.1)
    corr, _ = o3g.correspondences(empty, cuda(src), np.eye(4), 0.1)
    assert np.all(corr.cpu().numpy() == -1)
    grid = o3g.build_grid(cuda(tgt), 0.1)
    # empty source
    corr, _ = o3g.correspondences(grid, cuda(np.zeros((0, 3), np.float32)), np.eye(4), 0.1)
    assert corr.numel() == 0
    # a source far outside the grid's box, and a radius larger than the whole cloud
    far = np.array([[1e6, -1e6, 3e5], [0.0, 0.0, 0.0]], np.float32)
    corr, d2 = o3g.correspondences(grid, cuda(far), np.eye(4), 0.1)
    c_ref, d_ref = oracle.nn(far, tgt, 0.1)
    assert np.array_equal(corr.cpu().numpy(), c_ref)
    corr, d2 = o3g.correspondences(grid, cuda(src), np.eye(4), 5.0)
    c_ref, d_ref = oracle.nn(src, tgt, 5.0)
    assert np.array_equal(corr.cpu().numpy(), c_ref) and np.array_equal(d2.cpu().numpy(), d_ref)
    # strided rows (x, y, z, pad)
    src4 = np.zeros((50, 4), np.float32)
    src4[:, :3] = src
    corr4, d24 = o3g.correspondences(grid, cuda(src4), np.eye(4), 0.1)
    c_ref, d_ref = oracle.nn(src, tgt, 0.1)
    assert np.array_equal(corr4.cpu().numpy(), c_ref) and np.array_equal(d24.cpu().numpy(), d_ref)
    # every point in one cell (cell much larger than the cloud)
    big = o3g.build_grid(cuda(tgt), 100.0)
    corr, d2 = o3g.correspondences(big, cuda(src), np.eye(4), 0.3)
    c_ref, d_ref = oracle.nn(src, tgt, 0.3)
    assert np.array_equal(corr.cpu().numpy(), c_ref) and np.array_equal(d2.cpu().numpy(), d_ref)


def test_grid_with_far_outlier_enlarges_cells_and_stays_exact(o3g):
    g = synth.rng(6)
    tgt = g.uniform(-1, 1, (2000, 3)).astype(np.float32)
    tgt[17] = [5000.0, -3000.0, 2000.0]
    grid = o3g.build_grid(cuda(tgt), 0.05)
    n, cell = grid.info()
    assert n == 2000 and cell > 0.05
    src = g.uniform(-1, 1, (1000, 3)).astype(np.float32)
    corr, d2 = o3g.correspondences(grid, cuda(src), np.eye(4), 0.05)
    c_ref, d_ref = oracle.nn(src, tgt, 0.05)
    assert np.array_equal(corr.cpu().numpy(), c_ref) and np.array_equal(d2.cpu().numpy(), d_ref)


def test_nonfinite_input_rejected(o3g):
    tgt = np.zeros((10, 3), np.float32)
    tgt[3, 1] = np.nan
    with pytest.raises(o3g.O3GError) as e:
        o3g.build_grid(cuda(tgt), 0.1)
    assert e.value.status == o3g.ERR_NONFINITE


# ------------------------------------------------------------------- kNN


@pytest.mark.parametrize("n,radius,max_nn,cell", [(3000, 0.1, 30, 0.1), (2500, 0.2, 64, 0.07), (1200, 0.05, 1, 0.05),
                                                  (4001, 0.15, 7, 0.4)])
def test_knn_sets_bitexact(o3g, n, radius, max_nn, cell):
    g = synth.rng(n)
    pts = tie_cloud(g, n, -0.5, 0.5, quant=0.01)
    qry = np.vstack([pts[::3], g.uniform(-0.6, 0.6, (300, 3)).astype(np.float32)])
    grid = o3g.build_grid(cuda(pts), cell)
    idx, d2, cnt = o3g.knn_hybrid(grid, cuda(qry), radius, max_nn)
    i_ref, d_ref, c_ref = oracle.knn_hybrid(pts, qry, radius, max_nn)
    assert np.array_equal(cnt.cpu().numpy(), c_ref)
    assert np.array_equal(idx.cpu().numpy(), i_ref)
    assert np.array_equal(d2.cpu().numpy(), d_ref)


def test_knn_room_frame_sampled(o3g, room):
    grid = o3g.build_grid(cuda(room.tgt), 0.05)
    g = synth.rng(8)
    qry = room.tgt[np.sort(g.choice(len(room.tgt), 2000, replace=False))]
    idx, d2, cnt = o3g.knn_hybrid(grid, cuda(qry), 0.05, 30)
    i_ref, d_ref, c_ref = oracle.knn_hybrid(room.tgt, qry, 0.05, 30)
    assert np.array_equal(cnt.cpu().numpy(), c_ref)
    assert np.array_equal(idx.cpu().numpy(), i_ref)
    assert np.array_equal(d2.cpu().numpy(), d_ref)


def crowded_cloud(g):
    """A dense cube (thousands of points within the radius of every query, far more than a warp
    buffers), 700 copies of one point (keys that differ only by index, all at d2 = 0) and a
    cluster around that point."""
    cube = g.uniform(-0.05, 0.05, (3000, 3))
    copies = np.tile([[0.31, 0.32, 0.33]], (700, 1))
    near = np.array([0.31, 0.32, 0.33]) + g.uniform(-0.01, 0.01, (500, 3))
    pts = np.vstack([cube, near[:250], copies, near[250:]]).astype(np.float32)
    qry = np.vstack([pts[::13], pts[3250:3260], g.uniform(-0.06, 0.06, (100, 3)),
                     np.array([0.31, 0.32, 0.33]) + g.uniform(-0.012, 0.012, (100, 3))]).astype(np.float32)
    return pts, qry


@pytest.mark.parametrize("radius,max_nn", [(0.2, 30), (0.2, 32), (0.2, 1), (0.03, 30), (0.012, 7), (0.0, 30)])
def test_knn_crowded_neighbourhoods_bitexact(o3g, radius, max_nn):
    """More keys within the radius than the warp buffers (the buffer is cut to its max_nn smallest
    and later keys are filtered), hundreds of exactly tied distances (the selection's distance
    histogram puts them all in one bin), and radius 0 (only exact copies of the query qualify)."""
    pts, qry = crowded_cloud(synth.rng(41))
    grid = o3g.build_grid(cuda(pts), 0.1)
    idx, d2, cnt = o3g.knn_hybrid(grid, cuda(qry), radius, max_nn)
    i_ref, d_ref, c_ref = oracle.knn_hybrid(pts, qry, radius, max_nn)
    assert np.array_equal(cnt.cpu().numpy(), c_ref)
    assert np.array_equal(idx.cpu().numpy(), i_ref)
    assert np.array_equal(d2.cpu().numpy(), d_ref)
    assert c_ref.max() == max_nn or radius == 0.0


# --------------------------------------------------------------- normals


def unit_angle(a, b):
    """Angle between the lines of a and b (sign ignored), robust near 0 (atan2 of cross and dot)."""
    a = np.asarray(a, np.float64) / np.linalg.norm(a)
    b = np.asarray(b, np.float64) / np.linalg.norm(b)
    return math.atan2(np.linalg.norm(np.cross(a, b)), abs(float(a @ b)))


def check_normals(pts, n_gpu, radius, max_nn, viewpoint, sample=None):
    """Angle to the oracle's normal within a gap-scaled bound; orientation where it is well defined."""
    sample = np.arange(len(pts)) if sample is None else sample
    n_ora, ev = oracle.estimate_normals(pts, radius, max_nn, viewpoint=viewpoint, return_evals=True)
    idx, _, cnt = oracle.knn_hybrid(pts, pts[sample], radius, max_nn)
    worst = 0.0
    for row, i in enumerate(sample):
        ng = n_gpu[i].astype(np.float64)
        assert abs(np.linalg.norm(ng) - 1) < 1e-5
        if cnt[row] < 3:
            assert np.array_equal(n_gpu[i], [0, 0, 1])
            continue
        l0, l1, l2 = ev[i]
        X = pts[idx[row, : cnt[row]]].astype(np.float64)
        C = np.cov(X.T, bias=True)
        # any correct answer is (close to) a smallest eigenvector: Rayleigh quotient near lambda_0
        assert ng @ C @ ng <= l0 + 1e-5 * l2 + 1e-12
        if l1 - l0 > 1e-3 * l2:
            ang = unit_angle(ng, n_ora[i])
            bound = 2e-5 * l2 / (l1 - l0) + 2e-6
            worst = max(worst, ang / bound)
            assert ang <= bound, (i, ang, bound, ev[i])
            view = np.asarray(viewpoint, np.float64) - pts[i]
            facing = float(n_ora[i].astype(np.float64) @ view) / (np.linalg.norm(view) + 1e-30)
            if abs(facing) > 1e-3:
                assert np.sign(ng @ view) == np.sign(facing)
    return worst


def test_normals_sphere_plane(o3g):
    pr = synth.sphere_plane_pair()
    grid = o3g.build_grid(cuda(pr.tgt), 0.1)
    n_gpu = grid.estimate_normals(0.1, 30, viewpoint=(0.0, 0.0, 0.0)).cpu().numpy()
    check_normals(pr.tgt, n_gpu, 0.1, 30, (0.0, 0.0, 0.0))


def test_normals_room_frame_sampled(o3g, room):
    """Full-size RGB-D frame target (the bench's normal estimation), checked on a sample of points."""
    grid = o3g.build_grid(cuda(room.tgt), room.max_corr_dist)
    n_gpu = grid.estimate_normals(0.05, 30).cpu().numpy()
    g = synth.rng(9)
    sample = np.sort(g.choice(len(room.tgt), 1500, replace=False))
    n_ora_s = None  # the oracle computes all normals; sample the comparison only
    check_normals(room.tgt, n_gpu, 0.05, 30, (0.0, 0.0, 0.0), sample=sample)
    del n_ora_s


def test_normals_dense_cube(o3g):
    """Thousands of points within the radius of every point: the warp's key buffer is cut down to
    its 30 nearest several times before the neighbourhood is known."""
    pts = synth.rng(43).uniform(-0.05, 0.05, (3000, 3)).astype(np.float32)
    grid = o3g.build_grid(cuda(pts), 0.1)
    n_gpu = grid.estimate_normals(0.2, 30, viewpoint=(1.0, 0.0, 0.0)).cpu().numpy()
    check_normals(pts, n_gpu, 0.2, 30, (1.0, 0.0, 0.0))


def test_normals_degenerate_neighbourhoods(o3g):
    pts = np.array([[0, 0, 0], [0.01, 0, 0], [5, 5, 5], [5, 5, 5.001], [5, 5, 5.002]], np.float32)
    grid = o3g.build_grid(cuda(pts), 0.05)
    n_gpu = grid.estimate_normals(0.05, 30).cpu().numpy()
    assert np.array_equal(n_gpu[0], [0, 0, 1]) and np.array_equal(n_gpu[1], [0, 0, 1])
    # a line of three points: any unit vector normal to the line is a smallest eigenvector
    assert np.all(np.abs(n_gpu[2:, 2]) < 1e-3)


# --------------------------------------------------------- normal equations


def rel_errors(A, b, A_ref, b_ref, scale_b):
    ea = np.linalg.norm(A - A_ref) / np.linalg.norm(A_ref)
    eb = np.max(np.abs(b - b_ref)) / np.max(scale_b)
    return ea, eb


def oracle_equations(src, tgt, nrm, T, r):
    p = oracle.transform(src, T)
    corr, d2 = oracle.nn(p, tgt, r)
    A, b, sr2, sd2, cnt = oracle.normal_equations(p, tgt, nrm, corr, d2)
    m = corr >= 0
    J = np.zeros((m.sum(), 6))
    rr = np.zeros(m.sum())
    for k, i in enumerate(np.flatnonzero(m)):
        J[k], rr[k] = oracle.residual_jacobian(p[i], tgt[corr[i]], nrm[corr[i]])
    scale_b = np.abs(J).T @ np.abs(rr)
    return A, b, np.array([sr2, sd2, cnt]), scale_b


@pytest.mark.parametrize("which", ["sphere_plane", "room"])
def test_normal_equations_parity(o3g, which, room):
    if which == "sphere_plane":
        pr = synth.sphere_plane_pair()
        nrm = pr.tgt_nrm
        Ts = poses(11, 2, deg=5.0, trans=0.05) + [pr.T_gt]
        src = pr.src
    else:
        pr = room
        nrm = oracle.estimate_normals(pr.tgt, 0.05, 30)
        Ts = [np.eye(4), pr.T_gt]
        g = synth.rng(12)
        src = pr.src[np.sort(g.choice(len(pr.src), 20000, replace=False))]
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(nrm))
    for T in Ts:
        A, b, stats = o3g.normal_equations(grid, cuda(src), T, pr.max_corr_dist)
        A_ref, b_ref, st_ref, scale_b = oracle_equations(src, pr.tgt, nrm, T, pr.max_corr_dist)
        ea, eb = rel_errors(A, b, A_ref, b_ref, scale_b)
        assert ea <= 1e-5 and eb <= 1e-5, (ea, eb)
        assert np.array_equal(A, A.T)
        assert stats[2] == st_ref[2]
        assert stats[1] == pytest.approx(st_ref[1], rel=1e-5)
        assert stats[0] == pytest.approx(st_ref[0], rel=1e-5, abs=1e-12)


def test_normal_equations_sign_invariance(o3g):
    pr = synth.sphere_plane_pair(n=3000)
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(pr.tgt_nrm))
    A1, b1, _ = o3g.normal_equations(grid, cuda(pr.src), pr.T_gt, pr.max_corr_dist)
    flip = pr.tgt_nrm.copy()
    flip[::2] *= -1
    grid.set_normals(cuda(flip))
    A2, b2, _ = o3g.normal_equations(grid, cuda(pr.src), pr.T_gt, pr.max_corr_dist)
    assert np.array_equal(A1, A2) and np.array_equal(b1, b2)


@pytest.mark.parametrize("scale,offset", [(7.3, 0.0), (1e-3, 0.0), (1.0, 1000.0), (2.5, -40000.0)])
def test_normal_equations_scaled_normals_and_far_clouds(o3g, scale, offset):
    """The sums are accumulated in fixed point scaled by the target's coordinate box and the normals'
    length bound: normals that are not unit vectors and clouds far from the origin meet the oracle at
    the same bars (a bound taken too small would report non-finite sums)."""
    pr = synth.sphere_plane_pair(n=4000)
    tgt = (pr.tgt.astype(np.float64) + offset).astype(np.float32)
    src = (pr.src.astype(np.float64) + offset).astype(np.float32)
    nrm = (pr.tgt_nrm.astype(np.float64) * scale).astype(np.float32)
    r = pr.max_corr_dist
    grid = o3g.build_grid(cuda(tgt), r)
    grid.set_normals(cuda(nrm))
    shift = synth.make_T(np.eye(3), [0.004, -0.003, 0.002])
    for T in [np.eye(4), shift]:
        A, b, stats = o3g.normal_equations(grid, cuda(src), T, r)
        A_ref, b_ref, st_ref, scale_b = oracle_equations(src, tgt, nrm, T, r)
        assert st_ref[2] > 100
        ea, eb = rel_errors(A, b, A_ref, b_ref, scale_b)
        assert ea <= 1e-5 and eb <= 1e-5, (ea, eb)
        assert stats[2] == st_ref[2]
        assert stats[1] == pytest.approx(st_ref[1], rel=1e-5)


def test_nonfinite_normal_reported(o3g):
    """A NaN target normal that a correspondence uses makes the sums non-finite: both the normal
    equations and ICP report O3G_ERR_NONFINITE instead of returning a result."""
    pr = synth.sphere_plane_pair(n=2000)
    nrm = pr.tgt_nrm.copy()
    nrm[::50] = np.nan
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(nrm))
    with pytest.raises(o3g.O3GError) as e:
        o3g.normal_equations(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist)
    assert e.value.status == o3g.ERR_NONFINITE
    with pytest.raises(o3g.O3GError) as e:
        o3g.icp_point_to_plane_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, 5)
    assert e.value.status == o3g.ERR_NONFINITE
    # a non-finite normal that no correspondence uses changes nothing: the fixed-point scale takes the
    # largest finite normal length, and the result meets the oracle's
    tgt = np.vstack([pr.tgt, np.array([[50.0, 50.0, 50.0], [-50.0, 0.0, 0.0]], np.float32)])
    nrm2 = np.vstack([pr.tgt_nrm, np.array([[np.nan, 0.0, 1.0], [np.inf, 0.0, 0.0]], np.float32)])
    g2 = o3g.build_grid(cuda(tgt), pr.max_corr_dist)
    g2.set_normals(cuda(nrm2))
    res = o3g.icp_point_to_plane_grid(g2, cuda(pr.src), np.eye(4), pr.max_corr_dist, pr.max_iter)
    ref = oracle.icp_point_to_plane(pr.src, tgt, nrm2, np.eye(4), pr.max_corr_dist, pr.max_iter)
    assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
    ang, dt = synth.pose_error(res["T"], ref["T"])
    assert ang <= 1e-6 and dt <= 1e-6, (ang, dt)


# ------------------------------------------------------------------- ICP


def assert_pose_close(T, T_ref, tol=POSE_TOL):
    ang, dt = synth.pose_error(T, T_ref)
    assert ang <= tol and dt <= tol, (ang, dt)


def oracle_step(src, tgt, nrm, T, r, method="brute"):
    """One Gauss-Newton update of the oracle from pose T (Eq. 2), as a 4x4 FP64 pose.  method "grid" answers the
    correspondence step through the oracle's exact uniform grid, pinned bit-exact to the brute-force scan."""
    p = oracle.transform(src, T)
    corr, d2 = oracle.nn(p, tgt, r, method=method)
    A, b, _, _, cnt = oracle.normal_equations(p, tgt, nrm, corr, d2)
    xi, _ = oracle.ldlt_solve(A, b)
    return oracle.delta_T(xi) @ T, cnt


def gpu_trajectory(o3g, grid, src, r, K):
    """T_0 .. T_K of the GPU's own ICP run (each prefix rerun from the start; the GPU path is deterministic)."""
    out = [np.eye(4)]
    for k in range(1, K + 1):
        out.append(o3g.icp_point_to_plane_grid(grid, src, np.eye(4), r, k)["T"])
    return out


SHADOW_TOL = 1e-7


def assert_shadows_oracle(o3g, grid, src_np, tgt, nrm, r, K, method="brute", traj=None):
    """Every GPU iterate T_{k+1} is the oracle's Gauss-Newton step from the GPU's own T_k (within 1e-7).
    traj: the GPU's T_0 .. T_K when the caller already has them (else run on `grid`)."""
    if traj is None:
        traj = gpu_trajectory(o3g, grid, cuda(src_np), r, K)
    worst = 0.0
    for k in range(K):
        T_next, cnt = oracle_step(src_np, tgt, nrm, traj[k], r, method)
        ang, dt = synth.pose_error(traj[k + 1], T_next)
        worst = max(worst, ang, dt)
        assert ang <= SHADOW_TOL and dt <= SHADOW_TOL, (k, ang, dt)
    return traj, worst


def sensitivity(src, tgt, nrm, r, iters):
    """How far the oracle's own final pose moves when the initial pose moves by 1e-9 (rad and m)."""
    a = oracle.icp_point_to_plane(src, tgt, nrm, np.eye(4), r, iters)
    d = synth.make_T(synth.axis_angle_matrix([1.0, 2.0, 3.0], 1e-9), [1e-9, 0.0, 0.0])
    b = oracle.icp_point_to_plane(src, tgt, nrm, d, r, iters)
    return a, max(synth.pose_error(a["T"], b["T"]))


def test_icp_sphere_plane_matches_oracle(o3g):
    """Sphere-plus-plane pair: step-wise shadow of the oracle, and the end-to-end pose within the oracle's own
    sensitivity (the rotation about z is unobservable for this scene, so the map is ill-conditioned)."""
    pr = synth.sphere_plane_pair()
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(pr.tgt_nrm))
    assert_shadows_oracle(o3g, grid, pr.src, pr.tgt, pr.tgt_nrm, pr.max_corr_dist, pr.max_iter)
    res = o3g.icp_point_to_plane_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, pr.max_iter)
    ref, sens = sensitivity(pr.src, pr.tgt, pr.tgt_nrm, pr.max_corr_dist, pr.max_iter)
    assert res["status"] == ref["status"] and res["iters"] == ref["iters"]
    assert_pose_close(res["T"], ref["T"], tol=max(POSE_TOL, 20 * sens))
    # fitness and rmse (Sec. 3.3 result fields) against the oracle's evaluation at the GPU's own final pose
    ev = oracle.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, res["T"], pr.max_corr_dist, 0)
    assert res["fitness"] == ev["fitness"]
    assert res["rmse"] == pytest.approx(ev["rmse"], rel=1e-6)


def test_icp_room_frame_shadows_oracle(o3g, room):
    """RGB-D-frame pair at full size (both sides use the oracle's target normals): every one of the 30 GPU
    iterates the bench runs is the oracle's Gauss-Newton step from the previous GPU iterate."""
    nrm = oracle.estimate_normals(room.tgt, 0.05, 30)
    grid = o3g.build_grid(cuda(room.tgt), room.max_corr_dist)
    grid.set_normals(cuda(nrm))
    assert_shadows_oracle(o3g, grid, room.src, room.tgt, nrm, room.max_corr_dist, room.max_iter, method="grid")
    res = o3g.icp_point_to_plane_grid(grid, cuda(room.src), np.eye(4), room.max_corr_dist, room.max_iter)
    assert res["status"] == o3g.OK and res["iters"] == room.max_iter and res["fitness"] > 0.9
    ev = oracle.icp_point_to_plane(room.src, room.tgt, nrm, res["T"], room.max_corr_dist, 0)
    assert res["fitness"] == ev["fitness"]
    assert res["rmse"] == pytest.approx(ev["rmse"], rel=1e-6)


def _corner_scene(g, spacing=0.02):
    u = np.arange(0.0, 1.0, spacing)
    a, b = np.meshgrid(u, u)
    a, b = a.ravel(), b.ravel()
    z0 = np.zeros_like(a)
    P = [np.column_stack([a, b, z0]), np.column_stack([a, z0, b]), np.column_stack([z0, a, b])]
    N = [np.tile([0, 0, 1.0], (len(a), 1)), np.tile([0, 1.0, 0], (len(a), 1)), np.tile([1.0, 0, 0], (len(a), 1))]
    return np.vstack(P), np.vstack(N)


def test_icp_recovers_known_transform_noise_free(o3g):
    g = synth.rng(22)
    tgt, nrm = _corner_scene(g)
    T_gt = synth.perturbation(g, 2.0, 0.02)
    src = synth.apply_T(synth.inv_T(T_gt), tgt).astype(np.float32)
    grid = o3g.build_grid(cuda(tgt.astype(np.float32)), 0.05)
    grid.set_normals(cuda(nrm.astype(np.float32)))
    res = o3g.icp_point_to_plane_grid(grid, cuda(src), np.eye(4), 0.05, 30)
    assert_pose_close(res["T"], T_gt)
    assert res["fitness"] == 1.0 and res["rmse"] < 1e-6


def test_icp_is_deterministic(o3g):
    pr = synth.sphere_plane_pair(n=20000, seed=3)
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(pr.tgt_nrm))
    a = o3g.icp_point_to_plane_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, pr.max_iter)
    grid2 = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid2.set_normals(cuda(pr.tgt_nrm))
    b = o3g.icp_point_to_plane_grid(grid2, cuda(pr.src), np.eye(4), pr.max_corr_dist, pr.max_iter)
    assert np.array_equal(a["T"], b["T"]) and a["fitness"] == b["fitness"] and a["rmse"] == b["rmse"]


def test_icp_edge_cases(o3g):
    g = synth.rng(24)
    tgt = g.uniform(-1, 1, (100, 3)).astype(np.float32)
    nrm = np.tile(np.array([0, 0, 1], np.float32), (100, 1))
    grid = o3g.build_grid(cuda(tgt), 0.1)
    grid.set_normals(cuda(nrm))
    # far away: fewer than 6 correspondences
    res = o3g.icp_point_to_plane_grid(grid, cuda(tgt + 10), np.eye(4), 0.1, 10)
    ref = oracle.icp_point_to_plane(tgt + 10, tgt, nrm, np.eye(4), 0.1, 10)
    assert res["status"] == ref["status"] == o3g.WARN_FEW_CORR
    assert np.array_equal(res["T"], np.eye(4)) and res["iters"] == 0 and res["fitness"] == 0.0
    # max_iter = 0: evaluation only
    res = o3g.icp_point_to_plane_grid(grid, cuda(tgt), np.eye(4), 0.1, 0)
    assert res["status"] == o3g.OK and res["fitness"] == 1.0 and res["rmse"] == 0.0
    # empty source
    res = o3g.icp_point_to_plane_grid(grid, cuda(np.zeros((0, 3), np.float32)), np.eye(4), 0.1, 5)
    assert res["status"] == o3g.WARN_FEW_CORR and res["fitness"] == 0.0
    # planar target: frozen DOF, warning status, same pose as the oracle
    pl = np.column_stack([g.uniform(-1, 1, 800), g.uniform(-1, 1, 800), np.zeros(800)]).astype(np.float32)
    pn = np.tile(np.array([0, 0, 1], np.float32), (800, 1))
    src = (pl + np.array([0, 0, 0.01], np.float32)).astype(np.float32)
    gp = o3g.build_grid(cuda(pl), 0.1)
    gp.set_normals(cuda(pn))
    res = o3g.icp_point_to_plane_grid(gp, cuda(src), np.eye(4), 0.1, 5)
    ref = oracle.icp_point_to_plane(src, pl, pn, np.eye(4), 0.1, 5)
    assert res["status"] == ref["status"] == o3g.WARN_DEGENERATE
    assert_pose_close(res["T"], ref["T"])
    # non-finite pose
    bad = np.eye(4)
    bad[0, 3] = np.inf
    with pytest.raises(o3g.O3GError) as e:
        o3g.icp_point_to_plane_grid(grid, cuda(tgt), bad, 0.1, 3)
    assert e.value.status == o3g.ERR_NONFINITE
    # no normals on the grid
    g2 = o3g.build_grid(cuda(tgt), 0.1)
    with pytest.raises(o3g.O3GError):
        o3g.icp_point_to_plane_grid(g2, cuda(tgt), np.eye(4), 0.1, 3)


def test_icp_well_conditioned_end_to_end_within_1e6(o3g):
    """A noisy corner scene (all six DOF observable) run to convergence: final pose within 1e-6 of the oracle,
    same iteration count under the convergence threshold."""
    g = synth.rng(41)
    tgt, nrm = _corner_scene(g, spacing=0.01)
    T_gt = synth.perturbation(g, 3.0, 0.03)
    src = (synth.apply_T(synth.inv_T(T_gt), tgt) + g.normal(0, 0.002, tgt.shape)).astype(np.float32)
    tgt, nrm = tgt.astype(np.float32), nrm.astype(np.float32)
    grid = o3g.build_grid(cuda(tgt), 0.05)
    grid.set_normals(cuda(nrm))
    res = o3g.icp_point_to_plane_grid(grid, cuda(src), np.eye(4), 0.05, 100, eps=1e-7)
    ref = oracle.icp_point_to_plane(src, tgt, nrm, np.eye(4), 0.05, 100, eps=1e-7)
    assert ref["iters"] < 100 and res["iters"] == ref["iters"]
    assert_pose_close(res["T"], ref["T"])
    assert res["fitness"] == ref["fitness"]
    assert res["rmse"] == pytest.approx(ref["rmse"], rel=1e-6)


def test_one_shot_and_host_entry_points_agree(o3g):
    pr = synth.sphere_plane_pair(n=5000, seed=5)
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist)
    grid.set_normals(cuda(pr.tgt_nrm))
    a = o3g.icp_point_to_plane_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, pr.max_iter)
    b = o3g.icp_point_to_plane(cuda(pr.src), cuda(pr.tgt), cuda(pr.tgt_nrm), np.eye(4), pr.max_corr_dist,
                               pr.max_iter)
    c = o3g.register_point_to_plane_host(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter)
    assert np.array_equal(a["T"], b["T"]) and np.array_equal(a["T"], c["T"])
    assert a["fitness"] == b["fitness"] == c["fitness"]
    with pytest.raises(o3g.O3GError):
        o3g.icp_point_to_plane(cuda(pr.src), cuda(pr.tgt), cuda(pr.tgt_nrm[:-1]), np.eye(4), 0.05, 3)


def _same_result(a, b):
    assert a["status"] == b["status"] and a["iters"] == b["iters"]
    assert np.array_equal(a["T"], b["T"])
    assert a["fitness"] == b["fitness"] and a["rmse"] == b["rmse"]


def test_combined_entry_equals_separate_calls(o3g, room):
    """o3g_register_point_to_plane sorts the source on a side stream while the grid and normals are built; its
    result is the separate calls' (grid at 1.002 r, normals, ICP) bit for bit, with estimated or attached
    normals, with strided rows, and through the host-buffer entry that runs on it."""
    import torch
    r = room.max_corr_dist
    grid = o3g.build_grid(cuda(room.tgt), r * 1.002)
    grid.estimate_normals(0.05, 30, out=False)
    sep = o3g.icp_point_to_plane_grid(grid, cuda(room.src), np.eye(4), r, room.max_iter)
    comb = o3g.register_point_to_plane(cuda(room.src), cuda(room.tgt), None, np.eye(4), r, room.max_iter,
                                       normal_radius=0.05, normal_max_nn=30)
    _same_result(sep, comb)
    host = o3g.register_point_to_plane_host(room.src, room.tgt, None, np.eye(4), r, room.max_iter,
                                            normal_radius=0.05, normal_max_nn=30)
    _same_result(sep, host)
    # attached normals, 4-float rows, a pose and eps
    pr = synth.sphere_plane_pair(n=6000, seed=7)
    wide = lambda a: torch.from_numpy(np.hstack([a, np.ones((len(a), 1), np.float32)])).cuda()
    g2 = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist * 1.002)
    g2.set_normals(cuda(pr.tgt_nrm))
    T0 = synth.perturbation(synth.rng(8), 1.0, 0.01)
    sep2 = o3g.icp_point_to_plane_grid(g2, cuda(pr.src), T0, pr.max_corr_dist, 40, eps=1e-8)
    comb2 = o3g.register_point_to_plane(wide(pr.src), wide(pr.tgt), wide(pr.tgt_nrm), T0, pr.max_corr_dist, 40,
                                        eps=1e-8)
    _same_result(sep2, comb2)
    # empty source, non-finite source
    empty = o3g.register_point_to_plane(torch.zeros((0, 3), device="cuda"), cuda(pr.tgt), cuda(pr.tgt_nrm),
                                        np.eye(4), 0.05, 5)
    assert empty["status"] == o3g.WARN_FEW_CORR
    bad = pr.src.copy()
    bad[7, 2] = np.nan
    with pytest.raises(o3g.O3GError) as e:
        o3g.register_point_to_plane(cuda(bad), cuda(pr.tgt), cuda(pr.tgt_nrm), np.eye(4), 0.05, 5)
    assert e.value.status == o3g.ERR_NONFINITE


def test_host_entry_with_gpu_normals_matches_oracle_pipeline(o3g, room):
    """register_point_to_plane_host on the RGB-D-frame pair (GPU normals) against the oracle's pipeline."""
    res = o3g.register_point_to_plane_host(room.src, room.tgt, None, np.eye(4), room.max_corr_dist, room.max_iter,
                                           normal_radius=0.05, normal_max_nn=30)
    nrm = oracle.estimate_normals(room.tgt, 0.05, 30)
    ref = oracle.icp_point_to_plane(room.src, room.tgt, nrm, np.eye(4), room.max_corr_dist, room.max_iter)
    # GPU (float32) and oracle (float64) normals differ at rounding level and the 30-iteration trajectory of
    # this pair is sensitive (it has not converged), so the pipelines agree to a looser, stated bound
    ang, dt = synth.pose_error(res["T"], ref["T"])
    assert ang < 1e-3 and dt < 1e-3, (ang, dt)
    assert res["fitness"] == pytest.approx(ref["fitness"], abs=1e-3)


def test_combined_call_with_gpu_normals_shadows_oracle(o3g, room):
    """The call the bench times on the RGB-D-frame pair (o3g_register_point_to_plane: grid, GPU normals, ICP):
    the normals it uses are the separate calls' (bit for bit, tested above), downloaded here; with them, every
    one of its 30 iterates is the oracle's Gauss-Newton step from the previous iterate, and fitness / rmse are
    the oracle's evaluation at its final pose."""
    r = room.max_corr_dist
    grid = o3g.build_grid(cuda(room.tgt), r * 1.002)
    nrm = grid.estimate_normals(0.05, 30).cpu().numpy()
    src, tgt = cuda(room.src), cuda(room.tgt)
    traj, last = [np.eye(4)], None
    for k in range(1, room.max_iter + 1):
        last = o3g.register_point_to_plane(src, tgt, None, np.eye(4), r, k, normal_radius=0.05, normal_max_nn=30)
        traj.append(last["T"])
    assert_shadows_oracle(o3g, None, room.src, room.tgt, nrm, r, room.max_iter, method="grid", traj=traj)
    ev = oracle.icp_point_to_plane(room.src, room.tgt, nrm, last["T"], r, 0, nn_method="grid")
    assert last["fitness"] == ev["fitness"]
    assert last["rmse"] == pytest.approx(ev["rmse"], rel=1e-6)


@pytest.mark.parametrize("case", ["room", "ties", "sphere_plane"])
def test_warm_search_correspondence_set_bitexact(o3g, room, case):
    """The correspondence set at the final pose of an ICP run, found by the warm-started search the iterations
    use (the previous matches of the point and its warp neighbours as first candidates, then the grid search
    within that bound), bit-exact against the oracle at the GPU's own final pose: the full RGB-D-frame pair, a
    quantised cloud with exact ties and duplicate points, and the sphere-plane pair, after several iteration
    counts (0 = the cold search alone).  These pairs are below the size that keeps candidate lists; the next
    test covers those."""
    if case == "room":
        src, tgt, r = room.src, room.tgt, room.max_corr_dist
        nrm = oracle.estimate_normals(tgt, 0.05, 30)
        method = "grid"
    elif case == "ties":
        g = synth.rng(4321)
        tgt = tie_cloud(g, 6000, quant=0.01)
        # a moved copy, quantised again: many exactly equal distances, duplicate sources
        src = np.round(synth.apply_T(synth.perturbation(g, 2.0, 0.02), tgt[:5000]) / 0.01) * 0.01
        src = src.astype(np.float32)
        nrm = g.normal(size=tgt.shape)
        nrm = (nrm / np.linalg.norm(nrm, axis=1, keepdims=True)).astype(np.float32)
        r, method = 0.08, "brute"
    else:
        pr = synth.sphere_plane_pair()
        src, tgt, nrm, r, method = pr.src, pr.tgt, pr.tgt_nrm, pr.max_corr_dist, "brute"
    grid = o3g.build_grid(cuda(tgt), r * 1.002)
    grid.set_normals(cuda(nrm))
    d_src = cuda(src)
    for k in (0, 1, 2, 5, 30):
        res = o3g.icp_point_to_plane_grid(grid, d_src, np.eye(4), r, k, correspondences=True)
        p = oracle.transform(src, res["T"])
        c_ref, d_ref = oracle.nn(p, tgt, r, method=method)
        assert np.array_equal(res["corr"].cpu().numpy(), c_ref), (case, k)
        assert np.array_equal(res["d2"].cpu().numpy(), d_ref), (case, k)


def test_candidate_lists_on_quantised_pair_bitexact(o3g):
    """A pair large enough to keep candidate lists (at least 2^17 source points), with both clouds on a 2 mm
    lattice so that listed candidates often lie at exactly equal distances, and duplicated target points that
    tie at every distance: the correspondence set of the final evaluation after 0 to 40 iterations (no lists;
    lists built once the updates are small; rebuilt as points drift past their skin; held) is bit-exact against
    the oracle's search at the GPU's own final pose, and the fitness is its count."""
    pr = synth.sphere_plane_pair(n=160_000, seed=77)
    q = 0.002
    tgt = (np.round(pr.tgt / q) * q).astype(np.float32)
    nrm = pr.tgt_nrm.copy()
    tgt[80_000:90_000] = tgt[:10_000]  # later copies must lose every tie
    nrm[80_000:90_000] = nrm[:10_000]
    src = (np.round(pr.src / q) * q).astype(np.float32)
    r = pr.max_corr_dist
    assert len(src) >= 1 << 17
    grid = o3g.build_grid(cuda(tgt), r * 1.002)
    grid.set_normals(cuda(nrm))
    d_src = cuda(src)
    for k in (0, 4, 8, 12, 20, 40):
        res = o3g.icp_point_to_plane_grid(grid, d_src, np.eye(4), r, k, correspondences=True)
        p = oracle.transform(src, res["T"])
        c_ref, d_ref = oracle.nn(p, tgt, r, method="grid")
        assert np.array_equal(res["corr"].cpu().numpy(), c_ref), k
        assert np.array_equal(res["d2"].cpu().numpy(), d_ref), k
        assert res["fitness"] == float(np.count_nonzero(c_ref >= 0)) / len(c_ref)


def test_launch_forms_give_identical_results(o3g):
    """The latency and throughput forms of the iteration kernel differ only in stage size and occupancy: the
    correspondences are exact either way and the sums run in the same order, so results are bit-identical."""
    pr = synth.room_frame_pair()
    nrm = oracle.estimate_normals(pr.tgt, 0.05, 30)
    grid = o3g.build_grid(cuda(pr.tgt), pr.max_corr_dist * 1.002)
    grid.set_normals(cuda(nrm))
    cls = o3g.size_class((len(pr.src) + 127) // 128)
    out = []
    try:
        for cfg in (o3g.TILE_LATENCY, o3g.TILE_THROUGHPUT):
            o3g.set_tile_config(cls, cfg)
            assert o3g.get_tile_config(cls) == cfg
            out.append(o3g.icp_point_to_plane_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, 10))
            out.append(o3g.icp_point_to_point_grid(grid, cuda(pr.src), np.eye(4), pr.max_corr_dist, 5))
    finally:
        o3g.set_tile_config(cls, o3g.TILE_AUTO)
    assert np.array_equal(out[0]["T"], out[2]["T"]) and out[0]["rmse"] == out[2]["rmse"]
    assert np.array_equal(out[1]["T"], out[3]["T"]) and out[1]["fitness"] == out[3]["fitness"]
    with pytest.raises(o3g.O3GError):
        o3g.set_tile_config(40, 0)
