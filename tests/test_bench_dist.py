"""The benchmark's multi-GPU path is replicas only: every rank times its own
grid and the job reports the max over ranks.  The aggregation runs here as
two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, ws, port, q):
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=ws)
    try:
        local = [10.0 + rank, 100.0 - 5 * rank]
        out = bench.aggregate(ws, local, dist, "cpu")
        q.put((rank, out))
    finally:
        dist.destroy_process_group()


def test_replica_max_over_ranks():
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(ws):
        assert res[r] == [11.0, 100.0]


def test_single_rank_passthrough():
    import bench

    assert bench.aggregate(1, [3.0, 4.0]) == [3.0, 4.0]
