"""Multi-GPU runs of bench.py are independent replicas (one process per GPU, no data exchange):
the job time is the slowest rank's and the value counts every replica's node updates.  The
reduction is checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _worker(rank, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=2)
    import bench
    times = bench.replica_times([10.0 + 5.0 * rank, 7.0 - rank], 2)
    value = bench.replica_value(1000, 20, times[0] / 1e3, 2)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, times, value))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_report_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=30)
            if p.is_alive():
                p.terminate()
    assert [r for r, _, _ in res] == [0, 1]
    for _, times, value in res:
        assert times == [15.0, 7.0]
        assert value == pytest.approx(2 * 1000 * 20 / 0.015)


def test_one_replica_needs_no_process_group():
    import bench
    assert bench.replica_times([3.0, 4.0], 1) == [3.0, 4.0]
    assert bench.replica_value(10, 5, 2.0, 1) == 25.0
