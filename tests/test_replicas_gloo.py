"""The N > 1 path of bench.py on CPU: two gloo ranks (replicas) agree on the
slowest rank's time and the whole-job rate counts every rank's updates."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, ws, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = 10.0 * (rank + 1)                # rank 1 is the slow one
    m = bench.max_over_ranks(torch, ws, ms)
    rate = bench.job_rate(1e9, ws, m)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, m, rate))


def test_two_gloo_replicas():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, rate in out:
        assert m == pytest.approx(20.0)
        assert rate == pytest.approx(2 * 1e9 / 0.020)
