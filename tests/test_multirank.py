"""The multi-GPU form is independent replicas: each rank checks its own trace
and the job's throughput is all records over the slowest rank's time. The
aggregation runs here on CPU with two gloo ranks."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r checks (r + 1) million records in (r + 2) ms
        v, ms = bench.job_value((rank + 1) * 1_000_000, float(rank + 2), dist, "cpu")
        q.put((rank, v, ms))
    finally:
        dist.destroy_process_group()


def test_two_rank_replicas_aggregate_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=5) for _ in range(2))
    # all ranks agree: 3e6 records over the slowest rank's 3 ms = 1.0 Gev/s
    for _, v, ms in got:
        assert ms == pytest.approx(3.0)
        assert v == pytest.approx(1.0)


def test_single_process_value():
    import bench
    v, ms = bench.job_value(6_000_000, 2.0)
    assert (v, ms) == (pytest.approx(3.0), 2.0)
