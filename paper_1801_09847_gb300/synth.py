"""Seeded synthetic inputs shaped like the paper's registration workloads.

This module builds INPUTS only: point clouds, their analytic normals where the
scene has them, and ground-truth rigid transforms.  It contains none of the
registration method's arithmetic (no correspondence search, no residuals, no
normal estimation, no solve), so both the CUDA path and the oracle can be fed
from it without sharing any of the method.

The paper evaluates on RGB-D sequences and scene fragments (TUM, NYU, SUN3D,
Redwood, SceneNN; Sec. 3.1 and Sec. 3.4), none of which is available here.
The scenes below stand in for them with the same shapes: a sphere-plus-plane
object cloud, a 640x480 PrimeSense-intrinsics depth frame of a furnished room
(Sec. 3.1, ``PinholeCameraIntrinsic.prime_sense_default``), and batches of
uneven size.  All randomness is numpy PCG64 with a stated seed.
"""
from __future__ import annotations

import math
import os
import tempfile
from dataclasses import dataclass, field

import numpy as np

# PrimeSense default pinhole intrinsics: fx = fy = 525, cx = 319.5, cy = 239.5, 640 x 480.
PRIMESENSE = dict(width=640, height=480, fx=525.0, fy=525.0, cx=319.5, cy=239.5)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


# ----------------------------------------------------------------- poses


def axis_angle_matrix(axis, angle: float) -> np.ndarray:
    """Rotation matrix of `angle` radians about the unit `axis` (Rodrigues' formula)."""
    a = np.asarray(axis, np.float64)
    a = a / np.linalg.norm(a)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]], np.float64)
    return np.eye(3) + math.sin(angle) * K + (1.0 - math.cos(angle)) * (K @ K)


def make_T(R, t) -> np.ndarray:
    T = np.eye(4)
    T[:3, :3] = R
    T[:3, 3] = t
    return T


def inv_T(T) -> np.ndarray:
    R, t = T[:3, :3], T[:3, 3]
    return make_T(R.T, -R.T @ t)


def random_unit(g: np.random.Generator) -> np.ndarray:
    v = g.standard_normal(3)
    return v / np.linalg.norm(v)


def perturbation(g: np.random.Generator, deg: float, trans: float) -> np.ndarray:
    """A rigid motion: `deg` degrees about a random axis and a translation of length `trans`."""
    return make_T(axis_angle_matrix(random_unit(g), math.radians(deg)), trans * random_unit(g))


def apply_T(T, pts) -> np.ndarray:
    """Applies a 4x4 pose to N x 3 points in FP64 (input construction, not the method's FP32 transform)."""
    pts = np.asarray(pts, np.float64)
    return pts @ np.asarray(T)[:3, :3].T + np.asarray(T)[:3, 3]


def pose_error(Ta, Tb) -> tuple[float, float]:
    """(rotation angle in rad, translation distance) between two poses."""
    Ra, Rb = np.asarray(Ta)[:3, :3], np.asarray(Tb)[:3, :3]
    M = Ra @ Rb.T
    s = np.array([M[2, 1] - M[1, 2], M[0, 2] - M[2, 0], M[1, 0] - M[0, 1]])
    ang = math.atan2(np.linalg.norm(s) / 2.0, (np.trace(M) - 1.0) / 2.0)
    return abs(ang), float(np.linalg.norm(np.asarray(Ta)[:3, 3] - np.asarray(Tb)[:3, 3]))


# ------------------------------------------------------ sphere + plane scene


def sphere_plane(n: int, g: np.random.Generator):
    """n points on a unit sphere at the origin plus a 1 x 1 plane z = -1.5 (x, y in [-0.5, 0.5]).

    The split is area-proportional (4 pi : 1).  Returns FP64 points and their
    analytic unit normals (radial on the sphere, +z on the plane).
    """
    n_sph = int(round(n * 4.0 * math.pi / (4.0 * math.pi + 1.0)))
    n_pl = n - n_sph
    v = g.standard_normal((n_sph, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    pl = np.column_stack([g.uniform(-0.5, 0.5, n_pl), g.uniform(-0.5, 0.5, n_pl), np.full(n_pl, -1.5)])
    pts = np.vstack([v, pl])
    nrm = np.vstack([v, np.tile([0.0, 0.0, 1.0], (n_pl, 1))])
    return pts, nrm


@dataclass
class Pair:
    """One registration problem: source, target (FP32 N x 3), target normals, ground truth."""
    src: np.ndarray
    tgt: np.ndarray
    tgt_nrm: np.ndarray | None
    T_gt: np.ndarray
    max_corr_dist: float
    max_iter: int
    name: str = ""
    extra: dict = field(default_factory=dict)


def sphere_plane_pair(n: int = 4096, seed: int = 1, deg: float = 5.0, trans: float = 0.05,
                      noise: float = 0.002, max_corr_dist: float = 0.05, max_iter: int = 30) -> Pair:
    """Sphere-plus-plane pair: target with analytic normals; source = T_gt^-1 target + N(0, noise^2)."""
    g = rng(seed)
    tgt, nrm = sphere_plane(n, g)
    T_gt = perturbation(g, deg, trans)
    src = apply_T(inv_T(T_gt), tgt)
    if noise > 0:
        src = src + g.normal(0.0, noise, src.shape)
    return Pair(src.astype(np.float32), tgt.astype(np.float32), nrm.astype(np.float32), T_gt,
                max_corr_dist, max_iter, f"sphere_plane_n{n}_s{seed}")


# ------------------------------------------------------------ room ray-cast


@dataclass
class Room:
    half: float
    boxes_lo: np.ndarray  # (B, 3)
    boxes_hi: np.ndarray
    sph_c: np.ndarray  # (S, 3)
    sph_r: np.ndarray  # (S,)


def make_room(g: np.random.Generator, n_boxes: int = 20, n_spheres: int = 10, half: float = 2.0,
              keep_clear=((0.0, 0.0, 0.0),), clearance: float = 0.35) -> Room:
    """A [-half, half]^3 room with axis-aligned boxes (sides U(0.1, 0.6)) and spheres (r U(0.05, 0.3)).

    Objects are placed uniformly inside the room; a placement that would come
    within `clearance` of a point in `keep_clear` (camera centres) is redrawn.
    """
    clear = np.asarray(keep_clear, np.float64).reshape(-1, 3)
    lo_l, hi_l, c_l, r_l = [], [], [], []
    while len(lo_l) < n_boxes:
        side = g.uniform(0.1, 0.6, 3)
        c = g.uniform(-half + side / 2, half - side / 2)
        lo, hi = c - side / 2, c + side / 2
        d = np.linalg.norm(np.maximum(np.maximum(lo - clear, clear - hi), 0.0), axis=1)
        if np.all(d > clearance):
            lo_l.append(lo)
            hi_l.append(hi)
    while len(c_l) < n_spheres:
        r = g.uniform(0.05, 0.3)
        c = g.uniform(-half + r, half - r, 3)
        if np.all(np.linalg.norm(clear - c, axis=1) > r + clearance):
            c_l.append(c)
            r_l.append(r)
    return Room(half, np.array(lo_l), np.array(hi_l), np.array(c_l), np.array(r_l))


def _ray_cast(room: Room, origin: np.ndarray, dirs: np.ndarray) -> np.ndarray:
    """Distance along each (not necessarily unit) ray to the first surface."""
    o = origin[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / dirs
        # inside the room: exit distance through the walls
        t_wall = np.min(np.where(dirs > 0, (room.half - o) * inv, np.where(dirs < 0, (-room.half - o) * inv, np.inf)),
                        axis=1)
        best = t_wall.copy()
        for lo, hi in zip(room.boxes_lo, room.boxes_hi):
            t1 = (lo[None, :] - o) * inv
            t2 = (hi[None, :] - o) * inv
            tmin = np.max(np.minimum(t1, t2), axis=1)
            tmax = np.min(np.maximum(t1, t2), axis=1)
            hit = (tmax >= tmin) & (tmin > 1e-6)
            best = np.where(hit & (tmin < best), tmin, best)
        for c, r in zip(room.sph_c, room.sph_r):
            oc = o - c[None, :]
            a = np.sum(dirs * dirs, axis=1)
            b = 2.0 * np.sum(dirs * oc, axis=1)
            cc = np.sum(oc * oc) - r * r
            disc = b * b - 4 * a * cc
            sq = np.sqrt(np.maximum(disc, 0.0))
            t0 = (-b - sq) / (2 * a)
            hit = (disc >= 0) & (t0 > 1e-6)
            best = np.where(hit & (t0 < best), t0, best)
    return best


def depth_frame(room: Room, cam_to_world: np.ndarray, g: np.random.Generator, noise_k: float = 0.001,
                intr: dict = PRIMESENSE) -> np.ndarray:
    """A depth image (H x W, metres along the optical axis) ray-cast from a pinhole camera.

    Camera axes: x right, y down, z forward.  Depth noise N(0, (noise_k * z^2)^2).
    """
    W, H = intr["width"], intr["height"]
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    d_cam = np.stack([(u - intr["cx"]) / intr["fx"], (v - intr["cy"]) / intr["fy"], np.ones_like(u)], -1)
    d_cam = d_cam.reshape(-1, 3)
    d_world = d_cam @ cam_to_world[:3, :3].T
    t = _ray_cast(room, cam_to_world[:3, 3], d_world)  # d_cam.z == 1, so t is the depth
    z = t + g.normal(0.0, 1.0, t.shape) * noise_k * t * t
    return z.reshape(H, W)


def back_project(depth: np.ndarray, intr: dict = PRIMESENSE) -> np.ndarray:
    """create_point_cloud_from_rgbd_image's geometry (Sec. 3.1): pixels with finite positive depth to camera xyz."""
    H, W = depth.shape
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    ok = np.isfinite(depth) & (depth > 0)
    z = depth[ok]
    return np.column_stack([(u[ok] - intr["cx"]) * z / intr["fx"], (v[ok] - intr["cy"]) * z / intr["fy"], z])


def voxel_centroids(pts: np.ndarray, voxel: float) -> np.ndarray:
    """Input thinning as voxel_down_sample is commonly read (Fig. 1): one centroid per occupied voxel.

    Output order is by packed voxel key, which is deterministic for a given input.
    """
    keys = np.floor(pts / voxel).astype(np.int64)
    keys -= keys.min(axis=0)
    span = keys.max(axis=0) + 1
    lin = (keys[:, 0] * span[1] + keys[:, 1]) * span[2] + keys[:, 2]
    uniq, inv = np.unique(lin, return_inverse=True)
    cnt = np.bincount(inv, minlength=len(uniq)).astype(np.float64)
    out = np.empty((len(uniq), 3))
    for a in range(3):
        out[:, a] = np.bincount(inv, weights=pts[:, a], minlength=len(uniq)) / cnt
    return out


def room_frame_pair(seed: int = 2, deg: float = 3.0, trans: float = 0.05, voxel: float = 0.01,
                    max_corr_dist: float = 0.05, max_iter: int = 30) -> Pair:
    """RGB-D-frame-scale pair: two 640 x 480 depth frames of one furnished room.

    Camera 1 sits at the room centre looking +z (surfaces at about 2 m, where
    the depth noise stays below the voxel size and a frame thins to roughly
    60-100k points); camera 2 is camera 1 moved by a
    `deg` degree / `trans` m perturbation.  Each frame is back-projected into its
    own camera coordinates and voxel-thinned at `voxel` m.  Target = frame 1,
    source = frame 2; T_gt maps source (camera-2) coordinates to target
    (camera-1) coordinates.  Target normals are left to normal estimation.
    """
    g = rng(seed)
    room = make_room(g)
    cam1 = np.eye(4)
    P = perturbation(g, deg, trans)
    cam2 = cam1 @ P
    tgt = voxel_centroids(back_project(depth_frame(room, cam1, g)), voxel)
    src = voxel_centroids(back_project(depth_frame(room, cam2, g)), voxel)
    # shuffle so that the input order carries no spatial structure
    tgt = tgt[g.permutation(len(tgt))]
    src = src[g.permutation(len(src))]
    return Pair(src.astype(np.float32), tgt.astype(np.float32), None, P, max_corr_dist, max_iter,
                f"room_frame_s{seed}", extra=dict(viewpoint=(0.0, 0.0, 0.0)))


# ------------------------------------------------------- fused scene fragments


def _ray_cast_normals(room: Room, origin: np.ndarray, dirs: np.ndarray):
    """Distance along each ray to the first surface and that surface's unit normal (facing the camera)."""
    o = origin[None, :]
    n = len(dirs)
    ar = np.arange(n)
    with np.errstate(divide="ignore", invalid="ignore"):
        inv = 1.0 / dirs
        t_wall = np.where(dirs > 0, (room.half - o) * inv, np.where(dirs < 0, (-room.half - o) * inv, np.inf))
        ax = np.argmin(t_wall, axis=1)
        best = t_wall[ar, ax]
        nrm = np.zeros((n, 3))
        nrm[ar, ax] = -np.sign(dirs[ar, ax])
        for lo, hi in zip(room.boxes_lo, room.boxes_hi):
            t1 = (lo[None, :] - o) * inv
            t2 = (hi[None, :] - o) * inv
            t_near = np.minimum(t1, t2)
            axb = np.argmax(t_near, axis=1)  # the entry face
            tmin = t_near[ar, axb]
            tmax = np.min(np.maximum(t1, t2), axis=1)
            hit = (tmax >= tmin) & (tmin > 1e-6) & (tmin < best)
            best = np.where(hit, tmin, best)
            idx = np.nonzero(hit)[0]
            nrm[idx] = 0.0
            nrm[idx, axb[idx]] = -np.sign(dirs[idx, axb[idx]])
        a = np.sum(dirs * dirs, axis=1)
        for c, r in zip(room.sph_c, room.sph_r):
            oc = o[0] - c
            b = 2.0 * (dirs @ oc)
            cc = float(oc @ oc) - r * r
            disc = b * b - 4 * a * cc
            t0 = (-b - np.sqrt(np.maximum(disc, 0.0))) / (2 * a)
            hit = (disc >= 0) & (t0 > 1e-6) & (t0 < best)
            best = np.where(hit, t0, best)
            idx = np.nonzero(hit)[0]
            nrm[idx] = (o + t0[idx, None] * dirs[idx] - c[None, :]) / r
    return best, nrm


def pan_trajectory(count: int, radius: float, phase: float, pitch_deg: float) -> list:
    """Camera-to-world poses panning once around the room's vertical (y) axis.

    Camera k sits on a circle of `radius` about the centre, yawed by 2 pi k /
    count + phase and pitched by pitch_deg * sin(4 pi k / count), so the segment
    sees the walls all round plus parts of floor and ceiling.
    """
    poses = []
    for k in range(count):
        yaw = 2.0 * math.pi * k / count + phase
        pitch = math.radians(pitch_deg) * math.sin(4.0 * math.pi * k / count)
        R = axis_angle_matrix([0.0, 1.0, 0.0], yaw) @ axis_angle_matrix([1.0, 0.0, 0.0], pitch)
        poses.append(make_T(R, [radius * math.cos(yaw), 0.0, radius * math.sin(yaw)]))
    return poses


def _render_world(args):
    """One depth frame of a fused segment: world-frame points and analytic normals of its valid pixels."""
    room, cam_to_world, seed_words, noise_k, intr = args
    g = np.random.Generator(np.random.PCG64(np.random.SeedSequence(seed_words)))
    W, H = intr["width"], intr["height"]
    u, v = np.meshgrid(np.arange(W, dtype=np.float64), np.arange(H, dtype=np.float64))
    d_cam = np.stack([(u - intr["cx"]) / intr["fx"], (v - intr["cy"]) / intr["fy"], np.ones_like(u)], -1)
    d_cam = d_cam.reshape(-1, 3)
    R, t = cam_to_world[:3, :3], cam_to_world[:3, 3]
    depth, nrm = _ray_cast_normals(room, t, d_cam @ R.T)
    z = depth + g.normal(0.0, 1.0, depth.shape) * noise_k * depth * depth
    ok = np.isfinite(z) & (z > 0)
    return (d_cam[ok] * z[ok, None]) @ R.T + t, nrm[ok]


def voxel_centroids_normals(pts: np.ndarray, nrm: np.ndarray, voxel: float):
    """Fusion into a voxel grid: per occupied voxel the centroid of its points and the normalised mean of
    their analytic normals.  Output order is by packed voxel key."""
    keys = np.floor(pts / voxel).astype(np.int64)
    keys -= keys.min(axis=0)
    span = keys.max(axis=0) + 1
    lin = (keys[:, 0] * span[1] + keys[:, 1]) * span[2] + keys[:, 2]
    uniq, inv = np.unique(lin, return_inverse=True)
    cnt = np.bincount(inv, minlength=len(uniq)).astype(np.float64)
    c = np.empty((len(uniq), 3))
    m = np.empty((len(uniq), 3))
    for a in range(3):
        c[:, a] = np.bincount(inv, weights=pts[:, a], minlength=len(uniq)) / cnt
        m[:, a] = np.bincount(inv, weights=nrm[:, a], minlength=len(uniq))
    norm = np.linalg.norm(m, axis=1, keepdims=True)
    m = np.where(norm > 0, m / np.where(norm > 0, norm, 1.0), np.array([0.0, 0.0, 1.0]))
    return c, m


def fuse_segment(room: Room, poses: list, seed_words: tuple, voxel: float, noise_k: float = 0.001,
                 workers: int | None = None, intr: dict = PRIMESENSE):
    """Ray-cast every pose of a trajectory segment, move the points to world coordinates and fuse them at
    `voxel` m.  Frame k draws its depth noise from SeedSequence(seed_words + (k,)), so the result does not
    depend on `workers` (frames are rendered in a spawn-context process pool when workers > 1, which, as
    for any spawn pool, needs the calling script's top-level code behind ``if __name__ == "__main__":``)."""
    jobs = [(room, T, tuple(seed_words) + (k,), noise_k, intr) for k, T in enumerate(poses)]
    if workers is None:
        workers = min(16, len(jobs), os.cpu_count() or 1)
    if workers > 1:
        import concurrent.futures as cf
        import multiprocessing as mp
        with cf.ProcessPoolExecutor(workers, mp_context=mp.get_context("spawn")) as ex:
            frames = list(ex.map(_render_world, jobs))
    else:
        frames = [_render_world(j) for j in jobs]
    pts = np.concatenate([f[0] for f in frames])
    nrm = np.concatenate([f[1] for f in frames])
    return voxel_centroids_normals(pts, nrm, voxel)


def fragment_pair(n: int = 2_000_000, seed: int = 4, frames: int = 50, voxel: float = 0.005, deg: float = 1.0,
                  trans: float = 0.01, max_corr_dist: float = 0.02, max_iter: int = 50,
                  workers: int | None = None, cache: bool = True) -> Pair:
    """Scene-fragment pair: two fused fragments of one furnished room, `n` points each.

    Each fragment fuses `frames` 640 x 480 depth frames of a panning trajectory
    segment (pan_trajectory; segment 1 on a 0.30 m circle, segment 2 on a 0.35 m
    circle half a step out of phase, so the two sample the same surfaces
    differently) at `voxel` m, then keeps a seeded subset of exactly `n` voxels.
    Target = fragment 1 in world coordinates with its fused analytic normals;
    source = fragment 2 mapped by the inverse of T_gt (a `deg` degree / `trans` m
    perturbation), so T_gt maps source to target coordinates.  The result is
    cached in the system temp directory under a key of all parameters.
    """
    key = f"fragment_n{n}_s{seed}_f{frames}_v{voxel}_d{deg}_t{trans}"
    path = os.path.join(tempfile.gettempdir(), "o3g_synth_cache", key + ".npz")
    if cache and os.path.exists(path):
        z = np.load(path)
        src, tgt, nrm, T = z["src"], z["tgt"], z["nrm"], z["T"]
    else:
        g = rng(seed)
        seg1 = pan_trajectory(frames, 0.30, 0.0, 30.0)
        seg2 = pan_trajectory(frames, 0.35, math.pi / frames, 30.0)
        room = make_room(g, keep_clear=[T[:3, 3] for T in seg1 + seg2])
        T = perturbation(g, deg, trans)
        c1, n1 = fuse_segment(room, seg1, (seed, 1), voxel, workers=workers)
        c2, _ = fuse_segment(room, seg2, (seed, 2), voxel, workers=workers)
        if len(c1) < n or len(c2) < n:
            raise ValueError(f"fragments hold {len(c1)} and {len(c2)} voxels, fewer than {n}")
        k1 = g.choice(len(c1), n, replace=False)
        k2 = g.choice(len(c2), n, replace=False)
        tgt = c1[k1].astype(np.float32)
        nrm = n1[k1].astype(np.float32)
        src = apply_T(inv_T(T), c2[k2]).astype(np.float32)
        if cache:
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tmp = path + f".{os.getpid()}.npz"
            np.savez(tmp, src=src, tgt=tgt, nrm=nrm, T=T)
            os.replace(tmp, path)
    return Pair(src, tgt, nrm, T, max_corr_dist, max_iter, f"fragment_{n}_s{seed}",
                extra=dict(viewpoint=(0.0, 0.0, 0.0)))


# ------------------------------------------------------------------ batches


def log_uniform_sizes(count: int, lo: int, hi: int, g: np.random.Generator) -> np.ndarray:
    return np.exp(g.uniform(math.log(lo), math.log(hi), count)).astype(np.int64)


def sphere_plane_batch(count: int = 256, lo: int = 2000, hi: int = 200000, seed0: int = 1000,
                       size_seed: int = 3) -> list[Pair]:
    """`count` sphere-plus-plane pairs with log-uniform sizes in [lo, hi] and independent perturbations."""
    sizes = log_uniform_sizes(count, lo, hi, rng(size_seed))
    return [sphere_plane_pair(int(n), seed=seed0 + i) for i, n in enumerate(sizes)]
