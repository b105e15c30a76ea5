"""Benchmark: point-to-plane ICP registration on one GB300 per rank.

Headline (the default): the 2,000,000 x 2,000,000-point scene-fragment pair, the
largest single-GPU workload.  One step = the whole registration on the pair
already resident in HBM, through one o3g_register_point_to_plane call: build the
target grid, attach the fused target normals, 50 point-to-plane ICP iterations
(max_correspondence_distance 0.02 m) and the final fitness / rmse evaluation.
Metric: ICP point-pairs per second per iteration = N_source x iterations / step
time.  L2 is flushed (a 512 MiB write) before every step, outside the timed
events.  `e2e` repeats the measurement through the host-buffer entry point
(o3g_register_point_to_plane_host) with page-locked inputs, so the host-to-device
copies and the result read-back are inside the timed region.  The same line
carries the precision study (float32 + compensated sums against all-float64
terms, both against the float64 CPU oracle) and, nested under "nested", the
RGB-D-frame pair, the 256-pair batched call against the single-pair loop, and
the 1,000-request serving run (pairs/s, p50/p99 latency, iteration counts).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload fragment|rgbd_frame|batched|serving|p2p|voxel|ransac|normals_batch]

--impl reference times the CPU oracle (plain C, exact grid search, FP64 sums) on
the host cores on the headline workload: each step runs it on a seeded source
sample and scales the per-point iteration time to the whole source (the
per-pair set-up, its grid build and evaluation, is charged once per step).
Under torchrun every rank registers its own pair (independent problems, weak
scaling, no data-path collective); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ICP point-pairs/s per iteration"
UNIT = "point-pairs/s"
NORMAL_RADIUS, NORMAL_MAX_NN = 0.05, 30
L2_NOTE = "flushed (512 MiB write) before every step"
FRAGMENT_WORKLOAD = ("scene-fragment pair: two fused 50-frame fragments of a seeded room (20 boxes, 10 spheres, "
                     "4 m), 640x480 PrimeSense ray-cast depth, noise 0.001 z^2, 0.005 m voxels, seeded "
                     "2,000,000-point subsets, fused analytic normals; source moved 1 deg / 0.01 m; point-to-plane "
                     "ICP max_corr_dist 0.02, 50 iterations")
RGBD_WORKLOAD = ("RGB-D frame pair: seeded room (20 boxes, 10 spheres, 4 m), 640x480 PrimeSense ray-cast depth, "
                 "noise 0.001 z^2, 0.01 m voxel thinning; second frame moved 3 deg / 0.05 m; GPU normals "
                 "(radius 0.05, 30 NN); point-to-plane ICP max_corr_dist 0.05, 30 iterations")


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index
        self.path = None
        if shutil.which("nvidia-smi"):
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="o3g_clocks_", suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)

    def stop(self):
        if not self.proc:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def profiled_traffic(kernel_file: str, profile: str):
    """DRAM bytes per launch from a committed ncu summary, or None if the kernel source changed since."""
    import hashlib
    import re
    try:
        src = open(os.path.join(ROOT, "paper_1801_09847_gb300", "csrc", kernel_file), "rb").read()
        txt = open(os.path.join(ROOT, "profiles", profile)).read()
    except OSError:
        return None
    m_hash = re.search(r"source_sha256:\s*([0-9a-f]{16})", txt)
    m_bytes = re.search(r"dram_bytes_per_launch:\s*([0-9.]+)", txt)
    if not m_hash or not m_bytes or hashlib.sha256(src).hexdigest()[:16] != m_hash.group(1):
        return None
    return float(m_bytes.group(1))


def max_over_ranks(value: float, dist, dev) -> float:
    """The largest per-rank time: the job is as slow as its slowest rank."""
    import torch
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value: float, dist, dev) -> float:
    """Units processed by all ranks together (whole-job throughput numerator)."""
    import torch
    t = torch.tensor([float(value)], device=dev, dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())




def timed_steps(fn, steps, flush, stream, dist=None, dev=None, kinds=None):
    """CUDA-event time (ms, summed over `steps` calls of fn, L2 flushed before each, outside the events), the
    library's launch count over them, per-kernel device times (when `kinds` names instrumented kernels) and the
    last result.  Under torchrun the time is the maximum over ranks."""
    import torch

    from paper_1801_09847_gb300 import o3g
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    if kinds:
        o3g.timing_enable(True)
        for k in kinds.values():
            o3g.timing_read(k, reset=True)
    l0 = o3g.launch_count()
    total, out = 0.0, None
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    torch.cuda.synchronize()
    launches = o3g.launch_count() - l0
    kern = {}
    if kinds:
        o3g.timing_enable(False)
        for name, k in kinds.items():
            kern[name] = o3g.timing_read(k, reset=True)
    if dist:
        total = max_over_ranks(total, dist, dev)
    return total, launches, kern, out


def roofline_hbm(alg_bytes, kern_ms, kern_n, kernel, traffic=None):
    """HBM roofline of one kernel: algorithmic bytes per launch over its average CUDA-event launch time."""
    peak, which = peaks()
    avg_s = kern_ms / max(kern_n, 1) / 1e3
    achieved = alg_bytes / avg_s / 1e9 if avg_s > 0 else 0.0
    return {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kernel, "peak_source": which, "launches_timed": kern_n,
            "avg_launch_us": avg_s * 1e6, "algorithmic_bytes_per_launch": alg_bytes}


def icp_alg_bytes(ns, fitness):
    """Algorithmic bytes of one correspondence + reduction launch: the source xyz (12 B) of every point and the
    matched target xyz + normal (24 B) of every correspondence."""
    return ns * (12.0 + 24.0 * fitness)


def fragment_config(pr, iters):
    """The headline workload as both arms report it."""
    return {"workload": FRAGMENT_WORKLOAD, "n_source": int(len(pr.src)), "n_target": int(len(pr.tgt)),
            "iterations": int(iters), "max_corr_dist": float(pr.max_corr_dist), "l2": L2_NOTE,
            "parallelism": "replicas (one pair per rank)"}


def rgbd_config(pr, iters):
    return {"workload": RGBD_WORKLOAD, "n_source": int(len(pr.src)), "n_target": int(len(pr.tgt)),
            "iterations": int(iters), "max_corr_dist": float(pr.max_corr_dist), "normal_radius": NORMAL_RADIUS,
            "normal_max_nn": NORMAL_MAX_NN, "l2": L2_NOTE, "parallelism": "replicas (one pair per rank)"}


# ------------------------------------------------------- headline: scene fragments


def run_ours(args, ws, rank, local):
    """The 2M x 2M scene-fragment pair: float32 + compensated sums (the headline) and the all-float64 variant,
    both against the float64 CPU oracle; then the nested lines."""
    import torch

    from paper_1801_09847_gb300 import build, o3g, synth

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    # every rank registers its own copy of the pair (replicas); rank 0 renders it into the cache first, so
    # that the ranks of a node do not render it at once
    if dist and rank != 0:
        dist.barrier()
    pr = synth.fragment_pair(seed=4)
    if dist and rank == 0:
        dist.barrier()
    ns, nt, r, iters = len(pr.src), len(pr.tgt), pr.max_corr_dist, pr.max_iter
    src = torch.from_numpy(pr.src).to(dev)
    tgt = torch.from_numpy(pr.tgt).to(dev)
    nrm = torch.from_numpy(pr.tgt_nrm).to(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    init = np.eye(4)

    def step():
        # grid, attached normals and ICP in one call (the source sort overlaps the grid build)
        return o3g.register_point_to_plane(src, tgt, nrm, init, r, iters)

    def step_f64():
        g = o3g.build_grid(tgt, r * 1.002)
        g.set_normals(nrm)
        res = o3g.icp_point_to_plane_grid(g, src, init, r, iters, precision="f64")
        g.free()
        return res

    for _ in range(args.warmup):
        step()
    step_f64()
    icp_kind = {"icp": o3g.KERNEL_ICP_CORR, "grid": o3g.KERNEL_GRID}
    sampler = ClockSampler(local) if rank == 0 else None
    total_ms, launches, _, res = timed_steps(step, args.steps, flush, stream, dist, dev)
    clocks = sampler.stop() if sampler else None
    # a separate pass with per-launch CUDA events on the launching stream (kernel durations for the roofline)
    _, _, k32, _ = timed_steps(step, 3, flush, stream, kinds=icp_kind)
    f64_steps = max(3, args.steps // 4)
    ms64, _, _, res64 = timed_steps(step_f64, f64_steps, flush, stream, dist, dev)
    _, _, k64, _ = timed_steps(step_f64, 2, flush, stream, kinds=icp_kind)

    # e2e through the host-buffer entry point (page-locked inputs, copies and read-back inside the timed region)
    src_h = torch.from_numpy(pr.src).pin_memory()
    tgt_h = torch.from_numpy(pr.tgt).pin_memory()
    nrm_h = torch.from_numpy(pr.tgt_nrm).pin_memory()

    def step_host():
        return o3g.register_point_to_plane_host(src_h, tgt_h, nrm_h, init, r, iters)

    step_host()
    e2e_steps = max(3, args.steps // 2)
    e2e_ms, _, _, _ = timed_steps(step_host, e2e_steps, flush, stream, dist, dev)

    units = float(ns * res["iters"])
    if dist:
        units = sum_over_ranks(units, dist, dev)
    ms_step = total_ms / args.steps
    value = units / (ms_step / 1e3)
    if rank == 0:
        def roof(kern, result, traffic):
            ms, n = kern["icp"]
            return roofline_hbm(icp_alg_bytes(ns, result["fitness"]), ms, n, "k_icp_iter", traffic)

        # DRAM bytes per launch, averaged over one step's launches, from the committed capture of the float32
        # path (the all-float64 variant is a different kernel: no capture, no traffic figure)
        study = {"f32_compensated": {"ms_per_step": ms_step, "value": ns * res["iters"] / (ms_step / 1e3),
                                     "roofline": roof(k32, res, profiled_traffic("icp.cu", "k_icp_iter_fragment_2m.md")),
                                     "grid_ms": k32["grid"][0] / 3},
                 "f64": {"ms_per_step": ms64 / f64_steps, "value": ns * res64["iters"] / (ms64 / f64_steps / 1e3),
                         "roofline": roof(k64, res64, None)}}
        cpu = None
        if ws == 1 and not args.no_cpu_baseline:
            cpu = fragment_oracle_study(o3g, synth, pr, tgt, nrm, src, res, res64, study)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": fragment_config(pr, res["iters"]),
            "step": ("o3g_register_point_to_plane: grid build + attached normals + 50 ICP iterations + evaluation "
                     "(the source sort overlaps the grid build)"),
            "e2e": {"value": units / (e2e_ms / e2e_steps / 1e3), "unit": UNIT,
                    "h2d_bytes_per_step": (ns + 2 * nt) * 12, "d2h_bytes_per_step": 16 * 8 + 8 + 8 + 4,
                    "ms_per_step": e2e_ms / e2e_steps},
            "gpu_launches": launches,
            "roofline": study["f32_compensated"]["roofline"],
            "precision_study": study,
            "result": {"fitness": res["fitness"], "rmse": res["rmse"], "status": res["status"],
                       "iters": res["iters"]},
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        if ws == 1 and not args.no_nested:
            del src, tgt, nrm, src_h, tgt_h, nrm_h
            torch.cuda.empty_cache()
            line["nested"] = {"rgbd_frame": bench_rgbd(args, dev, flush, stream),
                              "batched": bench_batched(args, dev, flush, stream),
                              "serving": bench_serving(args)}
        print(json.dumps(line))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


def fragment_oracle_study(o3g, synth, pr, tgt, nrm, src, res32, res64, study):
    """The oracle (exact grid search, FP64 sums) on the whole fragment pair, timed on the host cores: the CPU
    baseline, and the reference for the pose, J^T J and J^T r errors of both GPU precisions."""
    import oracle
    oracle.build()
    threads = oracle.default_threads()
    ns, r, iters = len(pr.src), pr.max_corr_dist, pr.max_iter
    init = np.eye(4)
    t0 = time.perf_counter()
    ref = oracle.icp_point_to_plane(pr.src, pr.tgt, pr.tgt_nrm, init, r, iters, threads=threads, nn_method="grid")
    t_ora = time.perf_counter() - t0
    cpu = {"value": ns * ref["iters"] / t_ora, "unit": UNIT, "cores": threads, "kind": "oracle",
           "sample": (f"the whole pair: oracle ICP (exact uniform-grid correspondence search, FP64 sums) on all {ns} "
                      f"source points, {ref['iters']} iterations, {t_ora:.1f} s")}
    for key, res in (("f32_compensated", res32), ("f64", res64)):
        ang, dt = synth.pose_error(res["T"], ref["T"])
        study[key]["pose_error_vs_oracle"] = {"rad": ang, "m": dt}
        study[key]["iters"] = res["iters"]
    study["oracle"] = {"iters": ref["iters"], "fitness": ref["fitness"], "rmse": ref["rmse"],
                       "pose_error_vs_ground_truth": dict(zip(("rad", "m"), synth.pose_error(ref["T"], pr.T_gt)))}
    # J^T J and J^T r at the start pose and at the oracle's final pose
    g = o3g.build_grid(tgt, r * 1.002)
    g.set_normals(nrm)
    for label, T in (("start_pose", init), ("final_pose", ref["T"])):
        p = oracle.transform(pr.src, T)
        corr, d2 = oracle.nn(p, pr.tgt, r, threads=threads, method="grid")
        A_ref, b_ref, _, _, _ = oracle.normal_equations(p, pr.tgt, pr.tgt_nrm, corr, d2)
        m = corr >= 0
        pp = p[m].astype(np.float64)
        qn = pr.tgt_nrm[corr[m]].astype(np.float64)
        J = np.hstack([np.cross(pp, qn), qn])
        rr = np.sum((pp - pr.tgt[corr[m]].astype(np.float64)) * qn, axis=1)
        scale_b = np.abs(J).T @ np.abs(rr)
        for key, prec in (("f32_compensated", "f32"), ("f64", "f64")):
            A, b, _ = o3g.normal_equations(g, src, T, r, precision=prec)
            study[key][f"JtJ_rel_error_{label}"] = float(np.linalg.norm(A - A_ref) / np.linalg.norm(A_ref))
            study[key][f"Jtr_scaled_error_{label}"] = float(np.max(np.abs(b - b_ref)) / np.max(scale_b))
    g.free()
    return cpu


# ------------------------------------------------------------- RGB-D frame pair


def bench_rgbd(args, dev, flush, stream, rank=0):
    """The RGB-D-frame pair: grid + GPU normals + 30 iterations + evaluation in one call."""
    import torch

    from paper_1801_09847_gb300 import o3g, synth
    pr = synth.room_frame_pair(seed=2 + rank)
    ns = len(pr.src)
    src = torch.from_numpy(pr.src).to(dev)
    tgt = torch.from_numpy(pr.tgt).to(dev)
    init = np.eye(4)

    def step():
        return o3g.register_point_to_plane(src, tgt, None, init, pr.max_corr_dist, pr.max_iter,
                                           normal_radius=NORMAL_RADIUS, normal_max_nn=NORMAL_MAX_NN)

    for _ in range(args.warmup):
        step()
    kinds = {"icp_corr": o3g.KERNEL_ICP_CORR, "normals": o3g.KERNEL_NORMALS, "grid": o3g.KERNEL_GRID}
    total, launches, _, res = timed_steps(step, args.steps, flush, stream)
    _, _, kern, _ = timed_steps(step, 3, flush, stream, kinds=kinds)
    src_h = torch.from_numpy(pr.src).pin_memory()
    tgt_h = torch.from_numpy(pr.tgt).pin_memory()

    def step_host():
        return o3g.register_point_to_plane_host(src_h, tgt_h, None, init, pr.max_corr_dist, pr.max_iter,
                                                normal_radius=NORMAL_RADIUS, normal_max_nn=NORMAL_MAX_NN)

    step_host()
    e2e_ms, _, _, _ = timed_steps(step_host, args.steps, flush, stream)
    ms = total / args.steps
    units = ns * res["iters"]
    out = {"metric": METRIC, "value": units / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "config": rgbd_config(pr, res["iters"]),
           "step": "o3g_register_point_to_plane: grid build + GPU normals + 30 ICP iterations + evaluation",
           "e2e": {"value": units / (e2e_ms / args.steps / 1e3), "unit": UNIT,
                   "h2d_bytes_per_step": (ns + len(pr.tgt)) * 12, "d2h_bytes_per_step": 16 * 8 + 8 + 8 + 4,
                   "ms_per_step": e2e_ms / args.steps},
           "gpu_launches": launches,
           "roofline": roofline_hbm(icp_alg_bytes(ns, res["fitness"]), *kern["icp_corr"], "k_icp_iter",
                                    profiled_traffic("icp.cu", "k_icp_iter_room_frame_bench.md")),
           "kernels_ms_per_step": {k: v[0] / 3 for k, v in kern.items()},
           "result": {"fitness": res["fitness"], "rmse": res["rmse"], "status": res["status"]}}
    if not args.no_cpu_baseline:
        out["cpu_baseline"] = rgbd_cpu_baseline(pr)
    return out


def rgbd_cpu_sample(pr, n_sample: int, threads: int):
    """The oracle on the RGB-D pair: brute-force normals on the full target, then ICP (brute-force search) on a
    seeded source sample; returns (normals seconds, ICP seconds)."""
    import oracle
    from paper_1801_09847_gb300 import synth
    oracle.build()
    g = synth.rng(99)
    idx = np.sort(g.choice(len(pr.src), min(n_sample, len(pr.src)), replace=False))
    src = np.ascontiguousarray(pr.src[idx])
    t0 = time.perf_counter()
    nrm = oracle.estimate_normals(pr.tgt, NORMAL_RADIUS, NORMAL_MAX_NN, threads=threads)
    t1 = time.perf_counter()
    oracle.icp_point_to_plane(src, pr.tgt, nrm, np.eye(4), pr.max_corr_dist, pr.max_iter, threads=threads)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, len(src)


def rgbd_cpu_baseline(pr):
    import oracle
    threads = oracle.default_threads()
    n_sample = 49152
    t_nrm, t_icp, n_s = rgbd_cpu_sample(pr, n_sample, threads)
    # the ICP part scales with the sample; the target normals are paid once per pair
    per_pair_s = t_nrm + t_icp * len(pr.src) / n_s
    value = len(pr.src) * pr.max_iter / per_pair_s
    # the oracle's exact uniform-grid search on the whole pair (its pinned acceleration of the scan)
    nrm = oracle.estimate_normals(pr.tgt, NORMAL_RADIUS, NORMAL_MAX_NN, threads=threads)
    t0 = time.perf_counter()
    res = oracle.icp_point_to_plane(pr.src, pr.tgt, nrm, np.eye(4), pr.max_corr_dist, pr.max_iter, threads=threads,
                                    nn_method="grid")
    t_grid = time.perf_counter() - t0
    return {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"oracle normals on the full {len(pr.tgt)}-point target ({t_nrm:.2f} s) + oracle ICP on a "
                       f"seeded {n_s}-point source sample ({t_icp:.2f} s, {pr.max_iter} iterations), ICP time "
                       f"scaled to the full {len(pr.src)}-point source"),
            "grid_search": {"value": len(pr.src) * res["iters"] / (t_grid + t_nrm), "unit": UNIT,
                            "sample": (f"the whole pair: oracle normals ({t_nrm:.2f} s) + oracle ICP with its exact "
                                       f"uniform-grid correspondence search ({t_grid:.2f} s, {res['iters']} "
                                       f"iterations)")}}


# ---------------------------------------------------------- batched workload

FORM_NAMES = {0: "auto", 1: "latency", 2: "throughput"}
BATCH_WORKLOAD = ("256 sphere-plus-plane pairs, sizes log-uniform in 2k-200k points, independent seeds and "
                  "5 deg / 0.05 m perturbations, analytic target normals; point-to-plane ICP max_corr_dist 0.05, "
                  "30 iterations, all pairs in one batched call (one persistent launch per iteration, "
                  "graph-captured)")


def bench_batched(args, dev, flush, stream, rank=0):
    """Batched registrations against the plain single-pair loop on the same pairs (pairs/s, point-pairs/s)."""
    import torch

    from paper_1801_09847_gb300 import o3g, synth
    pairs = synth.sphere_plane_batch(args.batch_pairs, 2000, 200000, seed0=1000 + 100000 * rank)
    srcs = [torch.from_numpy(p.src).to(dev) for p in pairs]
    tgts = [torch.from_numpy(p.tgt).to(dev) for p in pairs]
    nrms = [torch.from_numpy(p.tgt_nrm).to(dev) for p in pairs]
    tune = None
    cell_factor = args.cell_factor
    if not args.no_autotune:
        from paper_1801_09847_gb300 import autotune
        tune = autotune.tune_batch(tgts, nrms, srcs, 0.05)
        cell_factor = tune["cell_factor"]
    grids = []
    for t, n in zip(tgts, nrms):
        g = o3g.build_grid(t, 0.05 * cell_factor)
        g.set_normals(n)
        grids.append(g)
    n_src = sum(len(p.src) for p in pairs)
    init = [np.eye(4)] * len(pairs)
    iters = pairs[0].max_iter

    def batched():
        return o3g.icp_point_to_plane_batch(grids, srcs, init, 0.05, iters)

    def single_loop():
        return [o3g.icp_point_to_plane_grid(g, s, np.eye(4), 0.05, iters) for g, s in zip(grids, srcs)]

    for _ in range(args.warmup):
        batched()
    single_loop()
    steps = max(3, args.steps // 2)
    ms_b, launches, _, res_b = timed_steps(batched, steps, flush, stream)
    ms_b /= steps
    s_steps = max(1, args.steps // 8)
    ms_s, _, _, res_s = timed_steps(single_loop, s_steps, flush, stream)
    ms_s /= s_steps
    # per-iteration kernel time from the instrumented graph launches
    _, _, kern, _ = timed_steps(batched, 2, flush, stream, kinds={"batch": o3g.KERNEL_ICP_BATCH})
    g_ms, g_n = kern["batch"]
    same = all(np.array_equal(a["T"], b["T"]) for a, b in zip(res_b, res_s))
    fit = float(np.mean([r["fitness"] for r in res_b]))
    alg = sum(icp_alg_bytes(len(p.src), rb["fitness"]) for p, rb in zip(pairs, res_b))
    # the plain loop as a user runs it: the library's automatic settings (the tuned points per thread suit a
    # full batch, not one small launch per pair); its poses meet the batch's within the pose tolerance
    if tune is not None:
        reset_tuning(tune)
    ms_p, _, _, res_p = timed_steps(single_loop, s_steps, flush, stream)
    ms_p /= s_steps
    from paper_1801_09847_gb300 import synth as _synth
    plain_err = max(max(_synth.pose_error(a["T"], b["T"])) for a, b in zip(res_b, res_p))
    for g in grids:
        g.free()
    return {
        "metric": METRIC, "value": n_src * iters / (ms_b / 1e3), "unit": UNIT, "ms_per_step": ms_b,
        "config": {"workload": BATCH_WORKLOAD, "pairs": len(pairs), "n_source_total": n_src, "iterations": iters,
                   "l2": L2_NOTE, "cell_factor": cell_factor},
        "autotune": tune and {k: v for k, v in tune.items() if k not in ("timings_ms", "ppt_timings_ms")} | {
            "ms_per_5_iteration_call": {f"cell {k[0]} r, {FORM_NAMES[k[1]]}": v for k, v in tune["timings_ms"].items()},
            "ms_per_5_iteration_call_by_points_per_thread": {f"pair class 2^{k[0]}, ppt {k[1]}": v
                                                             for k, v in tune["ppt_timings_ms"].items()}},
        "pairs_per_s": len(pairs) / (ms_b / 1e3),
        "single_pair_loop": {"ms_per_step": ms_p, "pairs_per_s": len(pairs) / (ms_p / 1e3),
                             "value": n_src * iters / (ms_p / 1e3), "settings": "automatic",
                             "max_pose_difference_to_batch": plain_err},
        "single_pair_loop_tuned_settings": {"ms_per_step": ms_s, "pairs_per_s": len(pairs) / (ms_s / 1e3),
                                            "results_bit_identical_to_batch": same},
        "speedup_vs_single_pair_loop": ms_p / ms_b,
        "gpu_launches": launches,
        "roofline": roofline_hbm(alg, g_ms / (iters + 1), g_n, "k_icp_iter (batched)"),
        "result": {"mean_fitness": fit, "statuses": sorted(set(r["status"] for r in res_b))},
    }


def reset_tuning(tune):
    """Back to the library's automatic launch form and points per thread after a tuned batch."""
    from paper_1801_09847_gb300 import o3g
    for c in tune["ppt"]:
        o3g.set_points_per_thread(c, 0)
    for c in range(32):
        o3g.set_tile_config(c, o3g.TILE_AUTO)


# ---------------------------------------------------------- serving workload

SERVE_WORKLOAD = ("registration requests, sphere-plus-plane pairs with sizes log-uniform in 5k-500k points, "
                  "Poisson arrivals, analytic target normals, point-to-plane ICP max_corr_dist 0.05 run to "
                  "convergence (max(|w|, |t|) < 1e-6, at most 100 iterations); continuous batching server")


def bench_serving(args, rank=0):
    """Open-loop serving: Poisson arrivals at fractions of the measured saturated rate; p50/p99 latency."""
    from paper_1801_09847_gb300 import o3g, synth
    g = synth.rng(5 + rank)
    sizes = synth.log_uniform_sizes(args.serve_requests, 5000, 500000, g)
    reqs = [synth.sphere_plane_pair(int(n), seed=20000 + 100000 * rank + k) for k, n in enumerate(sizes)]
    budget = int(args.serve_budget_gb * (1 << 30))

    def serve(arrivals):
        sv = o3g.Server(max_active=args.serve_slots, hbm_budget_bytes=budget)
        ids, done_at = {}, {}
        order = np.argsort(arrivals, kind="stable")
        nxt, n = 0, len(reqs)
        t0 = time.perf_counter()
        steps = 0
        while len(done_at) < n:
            now = time.perf_counter() - t0
            while nxt < n and arrivals[order[nxt]] <= now:
                k = int(order[nxt])
                pr = reqs[k]
                ids[sv.submit(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), 0.05, 100, eps=1e-6)] = k
                nxt += 1
            active, waiting, completed = sv.step()
            steps += 1
            if completed:
                t = time.perf_counter() - t0
                for rid in sv.completed():
                    done_at[ids[rid]] = (t, sv.poll(rid))
            elif active == 0 and waiting == 0 and nxt < n:
                time.sleep(max(0.0, min(1e-3, arrivals[order[nxt]] - (time.perf_counter() - t0))))
        elapsed = time.perf_counter() - t0
        sv.close()
        lat = np.array([done_at[k][0] - arrivals[k] for k in range(n)])
        it = np.array([done_at[k][1]["iters"] for k in range(n)])
        pts = sum(len(reqs[k].src) * done_at[k][1]["iters"] for k in range(n))
        return dict(elapsed_s=elapsed, pairs_per_s=n / elapsed, point_pairs_per_s=pts / elapsed,
                    p50_ms=float(np.percentile(lat, 50) * 1e3), p99_ms=float(np.percentile(lat, 99) * 1e3),
                    iterations={"mean": float(it.mean()), "min": int(it.min()), "p50": float(np.percentile(it, 50)),
                                "p90": float(np.percentile(it, 90)), "max": int(it.max()),
                                "converged_before_cap": int(np.sum(it < 100))},
                    host_steps=steps), {k: done_at[k][1] for k in range(n)}

    # saturated: every request waiting at t = 0
    sat, res_sat = serve(np.zeros(len(reqs)))
    out = {"saturated": sat}
    for frac in (0.5, 0.9):
        rate = frac * sat["pairs_per_s"]
        gaps = synth.rng(77).exponential(1.0 / rate, len(reqs))
        st, res = serve(np.cumsum(gaps) - gaps[0])
        st["arrival_rate_per_s"] = rate
        st["results_equal_saturated"] = all(np.array_equal(res[k]["T"], res_sat[k]["T"]) for k in res)
        out[f"poisson_{frac}"] = st
    # the plain single-request loop on the same requests
    t0 = time.perf_counter()
    single = [o3g.register_point_to_plane_host(pr.src, pr.tgt, pr.tgt_nrm, np.eye(4), 0.05, 100, eps=1e-6)
              for pr in reqs]
    t_single = time.perf_counter() - t0
    out["single_request_loop"] = {"pairs_per_s": len(reqs) / t_single,
                                  "results_equal_served": all(np.array_equal(a["T"], res_sat[k]["T"])
                                                              for k, a in enumerate(single))}
    out["saturated_speedup_vs_single_request_loop"] = sat["pairs_per_s"] / out["single_request_loop"]["pairs_per_s"]
    return {"metric": "served registrations/s (p50/p99 latency)", "value": out["poisson_0.9"]["pairs_per_s"],
            "unit": "pairs/s", "p50_ms": out["poisson_0.9"]["p50_ms"], "p99_ms": out["poisson_0.9"]["p99_ms"],
            "config": {"workload": SERVE_WORKLOAD, "requests": len(reqs), "slots": args.serve_slots,
                       "hbm_budget_gb": args.serve_budget_gb, "n_source_total": int(sum(sizes))},
            "serving": out}


def run_single(args, ws, rank, local):
    """One of the nested lines alone, printed as the line (development; single GPU)."""
    import torch

    from paper_1801_09847_gb300 import build
    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    sampler = ClockSampler(local)
    if args.workload == "rgbd_frame":
        out = bench_rgbd(args, dev, flush, stream)
    elif args.workload == "batched":
        out = bench_batched(args, dev, flush, stream)
    else:
        out = bench_serving(args)
    line = {"n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    line.update(out)
    line["clocks"] = sampler.stop()
    print(json.dumps(line))


# ------------------------------------------------- the rows after the ICP step

def _timed_steps(fn, steps, flush, stream):
    """Mean CUDA-event time (ms) of `steps` calls of fn, L2 flushed before each, and the last result."""
    import torch
    torch.cuda.synchronize()
    total, out = 0.0, None
    for _ in range(steps):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / steps, out


def _line(args, metric, value, unit, ms, workload, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": workload, "l2": "flushed (512 MiB write) before every step"}}
    line.update(extra)
    print(json.dumps(line))


def run_extra(args, ws, rank, local):
    """One line per row beyond the point-to-plane step: point-to-point ICP, voxel downsampling, RANSAC hypothesis
    validation, batched normals.  Single GPU (these rows are measured, not scaled)."""
    import torch

    import oracle
    from paper_1801_09847_gb300 import build, o3g, synth

    build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    peak, which = peaks()
    threads = oracle.default_threads()
    oracle.build()
    wl = args.workload
    l0 = o3g.launch_count()
    if wl == "p2p":
        pr = synth.room_frame_pair()
        src, tgt = torch.from_numpy(pr.src).to(dev), torch.from_numpy(pr.tgt).to(dev)

        def step():
            g = o3g.build_grid(tgt, pr.max_corr_dist * args.cell_factor)
            res = o3g.icp_point_to_point_grid(g, src, np.eye(4), pr.max_corr_dist, pr.max_iter)
            g.free()
            return res
        for _ in range(args.warmup):
            step()
        l0 = o3g.launch_count()
        ms, res = _timed_steps(step, args.steps, flush, stream)
        launches = o3g.launch_count() - l0
        o3g.timing_enable(True)
        o3g.timing_read(o3g.KERNEL_ICP_CORR, reset=True)
        _timed_steps(step, 3, flush, stream)
        o3g.timing_enable(False)
        k_ms, k_n = o3g.timing_read(o3g.KERNEL_ICP_CORR, reset=True)
        ns = len(pr.src)
        alg = ns * (12.0 + 12.0 * res["fitness"])
        avg_s = k_ms / max(k_n, 1) / 1e3
        g_sample = synth.rng(99)
        idx = np.sort(g_sample.choice(ns, 8192, replace=False))
        t0 = time.perf_counter()
        ref = oracle.icp_point_to_point(np.ascontiguousarray(pr.src[idx]), pr.tgt, np.eye(4), pr.max_corr_dist,
                                        pr.max_iter, threads=threads)
        t_ora = time.perf_counter() - t0
        _line(args, "ICP point-pairs/s per iteration (point-to-point)", ns * res["iters"] / (ms / 1e3), UNIT, ms,
              "RGB-D frame pair (as the headline line), point-to-point ICP (Horn's closed form), max_corr_dist 0.05, "
              "30 iterations; step = grid build + ICP + evaluation",
              {"gpu_launches": launches,
               "roofline": {"bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": alg / avg_s / 1e9 / peak, "traffic": None, "kernel": "k_icp_iter",
                            "peak_source": which, "avg_launch_us": avg_s * 1e6,
                            "algorithmic_bytes_per_launch": alg},
               "result": {"fitness": res["fitness"], "rmse": res["rmse"], "status": res["status"]},
               "cpu_baseline": {"value": len(idx) * ref["iters"] / t_ora, "unit": UNIT, "cores": threads,
                                "kind": "oracle", "sample": f"oracle point-to-point ICP on a seeded {len(idx)}-point "
                                                            f"source sample, {ref['iters']} iterations"}})
    elif wl == "voxel":
        g = synth.rng(2)
        room = synth.make_room(g)
        raw = synth.back_project(synth.depth_frame(room, np.eye(4), g)).astype(np.float32)
        pts = torch.from_numpy(raw).to(dev)
        for _ in range(args.warmup):
            o3g.voxel_down_sample(pts, 0.01)
        l0 = o3g.launch_count()
        ms, out = _timed_steps(lambda: o3g.voxel_down_sample(pts, 0.01), args.steps, flush, stream)
        launches = o3g.launch_count() - l0
        n, m = len(raw), int(out.shape[0])
        alg = 12.0 * n + 12.0 * m
        t0 = time.perf_counter()
        c_ref, _ = oracle.voxel_down_sample(raw, 0.01)
        t_ora = time.perf_counter() - t0
        same = bool(np.array_equal(out.cpu().numpy(), c_ref))
        _line(args, "voxel downsampling input points/s", n / (ms / 1e3), "points/s", ms,
              f"raw 640x480 ray-cast RGB-D frame ({n} points) thinned at 0.01 m ({m} voxels)",
              {"gpu_launches": launches,
               "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None,
                            "kernel": "whole o3g_voxel_down_sample call (coordinates, radix sort, heads, means)",
                            "peak_source": which, "algorithmic_bytes_per_call": alg},
               "result": {"voxels": m, "bit_identical_to_oracle": same},
               "cpu_baseline": {"value": n / t_ora, "unit": "points/s", "cores": 1, "kind": "oracle",
                                "sample": "oracle voxel downsampling of the whole frame (single thread)"}})
    elif wl == "ransac":
        pr = synth.room_frame_pair()
        src, tgt = torch.from_numpy(pr.src).to(dev), torch.from_numpy(pr.tgt).to(dev)
        grid = o3g.build_grid(tgt, pr.max_corr_dist * args.cell_factor)
        gh = synth.rng(140)
        poses = [pr.T_gt] + [synth.perturbation(gh, float(gh.uniform(0.5, 60)), float(gh.uniform(0.005, 0.5)))
                             @ pr.T_gt for _ in range(args.hypotheses - 1)]
        for _ in range(args.warmup):
            o3g.evaluate_poses(grid, src, poses, pr.max_corr_dist)
        l0 = o3g.launch_count()
        ms, (fit, rmse, cnt) = _timed_steps(lambda: o3g.evaluate_poses(grid, src, poses, pr.max_corr_dist),
                                            args.steps, flush, stream)
        launches = o3g.launch_count() - l0
        ns, H = len(pr.src), len(poses)
        alg = ns * H * 12.0 + float(np.sum(cnt)) * 12.0
        sub = poses[:4]
        t0 = time.perf_counter()
        f_ref, _, c_ref = oracle.evaluate_poses(pr.src, pr.tgt, sub, pr.max_corr_dist, threads=threads,
                                                nn_method="grid")
        t_ora = time.perf_counter() - t0
        _line(args, "hypothesis validation point evaluations/s", ns * H / (ms / 1e3), "point-evaluations/s", ms,
              f"RGB-D frame pair, {H} candidate poses (the true one and random 0.5-60 deg / 5-500 mm "
              f"perturbations of it), fitness + inlier rmse of all {ns} source points per pose, max_corr_dist 0.05",
              {"gpu_launches": launches, "hypotheses_per_s": H / (ms / 1e3),
               "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "kernel": "k_eval_poses",
                            "peak_source": which, "algorithmic_bytes_per_call": alg},
               "result": {"best_pose": int(np.argmax(fit)), "best_fitness": float(np.max(fit)),
                          "counts_equal_oracle_first4": bool(np.array_equal(cnt[:4], c_ref))},
               "cpu_baseline": {"value": ns * len(sub) / t_ora, "unit": "point-evaluations/s", "cores": threads,
                                "kind": "oracle", "sample": f"oracle evaluation (exact grid search) of the first "
                                                            f"{len(sub)} poses on the whole source"}})
    elif wl == "normals_batch":
        pairs = synth.sphere_plane_batch(args.batch_pairs, 2000, 200000, seed0=1000)
        tgts = [torch.from_numpy(p.tgt).to(dev) for p in pairs]
        grids = [o3g.build_grid(t, 0.1) for t in tgts]

        def batched():
            o3g.estimate_normals_batch(grids, 0.1, 30)

        def loop():
            for g in grids:
                g.estimate_normals(0.1, 30, out=False)
        for _ in range(args.warmup):
            batched()
            loop()
        l0 = o3g.launch_count()
        ms, _ = _timed_steps(batched, args.steps, flush, stream)
        launches = o3g.launch_count() - l0
        ms_loop, _ = _timed_steps(loop, max(1, args.steps // 2), flush, stream)
        n = sum(len(p.tgt) for p in pairs)
        alg = 24.0 * n
        sample = pairs[0].tgt
        t0 = time.perf_counter()
        oracle.estimate_normals(sample, 0.1, 30, threads=threads)
        t_ora = time.perf_counter() - t0
        _line(args, "normal estimation points/s (batched)", n / (ms / 1e3), "points/s", ms,
              f"{len(pairs)} sphere-plus-plane clouds (log-uniform 2k-200k points, {n} in all), hybrid radius 0.1, "
              f"30 neighbours, all in one launch",
              {"gpu_launches": launches,
               "one_launch_per_cloud": {"ms_per_step": ms_loop, "value": n / (ms_loop / 1e3)},
               "roofline": {"bound": "hbm", "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                            "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "kernel": "k_normals_batch",
                            "peak_source": which, "algorithmic_bytes_per_call": alg},
               "cpu_baseline": {"value": len(sample) / t_ora, "unit": "points/s", "cores": threads, "kind": "oracle",
                                "sample": f"oracle normals (brute force) of the first cloud ({len(sample)} points)"}})


# ------------------------------------------------------- reference arm: the oracle


def fragment_cpu_sample(pr, n_sample: int, threads: int, seed: int):
    """The oracle on the fragment pair for a seeded source sample: a zero-iteration call (the per-pair set-up:
    its grid over the target and one evaluation pass) and the full 50-iteration call; returns (set-up seconds,
    sample size, iterations, seconds of the full call)."""
    import oracle
    from paper_1801_09847_gb300 import synth
    g = synth.rng(seed)
    idx = np.sort(g.choice(len(pr.src), min(n_sample, len(pr.src)), replace=False))
    src = np.ascontiguousarray(pr.src[idx])
    t0 = time.perf_counter()
    oracle.icp_point_to_plane(src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, 0, threads=threads,
                              nn_method="grid")
    t1 = time.perf_counter()
    res = oracle.icp_point_to_plane(src, pr.tgt, pr.tgt_nrm, np.eye(4), pr.max_corr_dist, pr.max_iter,
                                    threads=threads, nn_method="grid")
    t2 = time.perf_counter()
    return t1 - t0, len(src), res["iters"], t2 - t1


def run_reference(args, ws, rank, local):
    """The oracle on the headline workload, each step a bounded sample whose ICP time is scaled to the whole
    source; the per-pair set-up (grid build and evaluation) is charged once per step."""
    if rank != 0:
        return
    import oracle
    from paper_1801_09847_gb300 import synth
    oracle.build()
    threads = oracle.default_threads()
    pr = synth.fragment_pair(seed=4)
    ns = len(pr.src)
    n_sample = args.ref_sample
    for w in range(args.warmup):
        fragment_cpu_sample(pr, 256, threads, 500 + w)
    step_s, units, iters = [], 0.0, pr.max_iter
    for k in range(args.steps):
        t_setup, n_s, iters, t_full = fragment_cpu_sample(pr, n_sample, threads, 600 + k)
        # t_full holds one set-up (grid + evaluation) and the iterations over the sample
        t_iter = max(t_full - t_setup, 0.0)
        step_s.append(t_setup + t_iter * ns / n_s)
        units += ns * iters
    total = sum(step_s)
    value = units / total
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total / args.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": fragment_config(pr, iters),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": (f"each step: the oracle (exact uniform-grid search, FP64 sums) on a seeded "
                                    f"{n_sample}-point source sample against the whole {len(pr.tgt)}-point target, "
                                    f"{iters} iterations; its iteration time scaled to all {ns} source points, "
                                    f"plus the per-pair set-up (grid build and evaluation) once")},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["fragment", "rgbd_frame", "batched", "serving", "p2p", "voxel", "ransac",
                                           "normals_batch"], default="fragment",
                    help="fragment: the headline line (2M x 2M scene fragments, precision study, and the RGB-D, "
                         "batched and serving lines nested); rgbd_frame, batched, serving: one nested line alone; "
                         "p2p, voxel, ransac, normals_batch: the rows after the point-to-plane step")
    ap.add_argument("--no-nested", action="store_true", help="fragment: skip the nested lines")
    ap.add_argument("--serve-requests", type=int, default=1000)
    ap.add_argument("--serve-slots", type=int, default=256)
    ap.add_argument("--serve-budget-gb", type=float, default=64.0)
    ap.add_argument("--batch-pairs", type=int, default=256)
    ap.add_argument("--hypotheses", type=int, default=1000, help="ransac: candidate poses per call")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true", help="batched: skip the tuning")
    ap.add_argument("--ref-sample", type=int, default=65536, help="reference arm: source points per step")
    ap.add_argument("--cell-factor", type=float, default=1.002, help="grid cell = factor x max_corr_dist")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank, local)
    elif args.workload == "fragment":
        run_ours(args, ws, rank, local)
    elif args.workload in ("rgbd_frame", "batched", "serving"):
        if rank == 0:
            run_single(args, ws, rank, local)
    elif rank == 0:
        run_extra(args, ws, rank, local)


if __name__ == "__main__":
    main()
