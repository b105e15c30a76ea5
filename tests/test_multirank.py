"""The bench's multi-rank path on CPU: 2 gloo ranks, independent problems, max-over-ranks time (no GPU)."""
from __future__ import annotations

import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port() -> int:
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    from paper_1801_09847_gb300 import synth
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench.dist_env()
    assert (ws, r, local) == (world, rank, rank)
    # each rank registers its own problem (weak scaling): different seeds, same size class
    pr = synth.sphere_plane_pair(n=1000, seed=2 + rank)
    units = len(pr.src) * pr.max_iter
    ms = 10.0 + 5.0 * rank               # a stand-in per-rank time
    out[rank] = (bench.max_over_ranks(ms, dist, torch.device("cpu")),
                 bench.sum_over_ranks(units, dist, torch.device("cpu")), float(pr.src[0, 0]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_aggregate_like_the_bench():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                  # max over ranks
    assert res[0][1] == res[1][1] == 2 * 1000 * 30         # whole-job units
    assert res[0][2] != res[1][2]                          # ranks work on different problems
