"""Multi-rank path of bench.py on CPU (gloo, world size 2): each rank checks
its own replica, the job's value is all ranks' ops over the slowest rank's
time (replicas only: no data exchange)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [10.0, 25.0][rank]
    ops_local = [1000, 1000][rank]
    value, ms, total = bench.aggregate(ms_local, ops_local, world, device="cpu")
    q.put((rank, value, ms, total))
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, total in res:
        assert ms == 25.0
        assert total == 2000
        assert value == pytest.approx(2000 / 0.025)
