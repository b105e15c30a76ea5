"""Serving loop (continuous batching): every request's result equals the single-request result (GPU)."""
from __future__ import annotations

import numpy as np
import pytest

from paper_1801_09847_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def o3g():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1801_09847_gb300 import build, o3g as mod
    build.build()
    mod.lib()
    return mod


@pytest.fixture(scope="module")
def requests():
    reqs = []
    for k, n in enumerate([3000, 500, 12000, 40000, 7000]):
        pr = synth.sphere_plane_pair(n=n, seed=700 + k)
        reqs.append(dict(src=pr.src, tgt=pr.tgt, tgt_nrm=pr.tgt_nrm, max_iter=25, eps=0.0))
    pr = synth.sphere_plane_pair(n=6000, seed=777, noise=0.0005)
    reqs.append(dict(src=pr.src, tgt=pr.tgt, tgt_nrm=None, max_iter=100, eps=1e-6))   # GPU normals, convergence
    reqs.append(dict(src=(pr.src + 30).astype(np.float32), tgt=pr.tgt, tgt_nrm=pr.tgt_nrm, max_iter=10, eps=0.0))
    reqs.append(dict(src=np.zeros((0, 3), np.float32), tgt=pr.tgt, tgt_nrm=pr.tgt_nrm, max_iter=5, eps=0.0))
    reqs.append(dict(src=pr.src, tgt=pr.tgt, tgt_nrm=pr.tgt_nrm, max_iter=0, eps=0.0))
    return reqs


def alone(o3g, rq):
    return o3g.register_point_to_plane_host(rq["src"], rq["tgt"], rq["tgt_nrm"], np.eye(4), 0.05, rq["max_iter"],
                                            eps=rq["eps"], normal_radius=0.1, normal_max_nn=30)


def serve(o3g, reqs, max_active, budget, arrivals=None):
    sv = o3g.Server(max_active=max_active, hbm_budget_bytes=budget)
    ids, results, peak_active = {}, {}, 0
    arrivals = arrivals or [0] * len(reqs)
    step = 0
    while len(results) < len(reqs):
        for k, rq in enumerate(reqs):
            if k not in ids and arrivals[k] <= step:
                ids[k] = sv.submit(rq["src"], rq["tgt"], rq["tgt_nrm"], np.eye(4), 0.05, rq["max_iter"], eps=rq["eps"],
                                   normal_radius=0.1, normal_max_nn=30)
        active, waiting, done = sv.step()
        peak_active = max(peak_active, active)
        for k, rid in ids.items():
            if k not in results:
                r = sv.poll(rid)
                if r is not None:
                    results[k] = r
        step += 1
        assert step < 10000
    sv.close()
    return [results[k] for k in range(len(reqs))], peak_active


def _same(a, b):
    assert a["status"] == b["status"] and a["iters"] == b["iters"]
    assert np.array_equal(a["T"], b["T"])
    assert a["fitness"] == b["fitness"] and a["rmse"] == b["rmse"]


def test_served_results_equal_alone(o3g, requests):
    ref = [alone(o3g, rq) for rq in requests]
    got, peak = serve(o3g, requests, max_active=3, budget=8 << 30)
    assert peak <= 3
    for a, b in zip(ref, got):
        _same(a, b)
    assert got[5]["iters"] < 100                        # converged under eps
    assert got[6]["status"] == o3g.WARN_FEW_CORR and got[7]["status"] == o3g.WARN_FEW_CORR
    assert got[8]["iters"] == 0


def test_staggered_arrivals_and_tight_budget(o3g, requests):
    ref = [alone(o3g, rq) for rq in requests]
    got, _ = serve(o3g, requests, max_active=64, budget=8 << 30, arrivals=[0, 3, 3, 7, 8, 20, 21, 40, 41])
    for a, b in zip(ref, got):
        _same(a, b)
    # a budget below any two requests together (but above each one alone) serves them one by one
    sub = requests[:3]
    sizes = sorted(_bytes(rq) for rq in sub)
    budget = sizes[0] + sizes[1] - 1
    assert sizes[-1] <= budget
    got1, peak1 = serve(o3g, sub, max_active=8, budget=budget)
    assert peak1 == 1
    for a, b in zip(ref[:3], got1):
        _same(a, b)


def _bytes(rq):
    from paper_1801_09847_gb300 import o3g
    return o3g.Server.request_bytes(len(rq["src"]), len(rq["tgt"]))


def test_server_errors(o3g, requests):
    sv = o3g.Server(max_active=2, hbm_budget_bytes=1 << 20)
    with pytest.raises(o3g.O3GError) as e:
        sv.submit(requests[3]["src"], requests[3]["tgt"], requests[3]["tgt_nrm"])
    assert e.value.status == o3g.ERR_OOM
    with pytest.raises(o3g.O3GError):
        sv.poll(12345)
    sv.close()
