"""bench.py's multi-rank path on CPU: two gloo ranks, the same init, barrier
and max / sum over ranks that the benchmark uses for N independent replicas
(one per GPU; value = all ranks' DOF-updates / max time over ranks)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    import bench
    import torch.distributed as dist
    w, r, loc = bench.dist_init(False)
    ms = bench.max_over_ranks(w, 10.0 * (r + 1))
    dof = bench.sum_over_ranks(w, 1000.0 * (r + 1))
    bench.barrier(w)
    q.put((r, w, ms, dof))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, w, ms, dof in out:
        assert w == 2
        assert ms == 20.0      # max over ranks of the timed region
        assert dof == 3000.0   # units processed by all ranks
