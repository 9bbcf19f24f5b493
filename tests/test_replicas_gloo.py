"""Multi-GPU in bench.py means independent replicas (no data-path collective): the whole-job
value is the units of all ranks over the slowest rank's time.  The reduction is checked here on
two CPU processes over gloo (127.0.0.1)."""
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
    try:
        local_ms = [40.0, 50.0][rank]          # rank 1 is the slowest
        value, ms = bench._replica_value(1000, local_ms, dist, world, "cpu")
        total = bench._reduce(float(rank + 1), dist, "cpu", "sum")
        q.put((rank, value, ms, total))
    finally:
        dist.destroy_process_group()


def test_replica_throughput_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, total in got:
        assert ms == 50.0
        assert value == pytest.approx(2 * 1000 / 0.050)
        assert total == 3.0


def test_single_process_needs_no_collective():
    import bench
    assert bench._replica_value(10, 20.0, None, 1, "cpu") == (500.0, 20.0)
    assert bench._reduce(7.0, None, "cpu", "sum") == 7.0
