"""The benchmark's N > 1 aggregation on CPU: two gloo ranks run independent replicas; the job
time is the slowest rank's and the throughput counts every rank's evaluations."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 100.0 + 50.0 * rank  # rank 1 is slower
    slow = bench.slowest_rank_ms(local_ms, dist, "cpu")
    out[rank] = (slow, bench.job_throughput(200, world, slow))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_aggregate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        slow, thr = out[r]
        assert slow == 150.0
        assert abs(thr - 2 * 200 / 0.150) < 1e-9


def test_single_rank_needs_no_collective():
    import bench
    assert bench.slowest_rank_ms(12.5, None, "cpu") == 12.5
    assert bench.job_throughput(10, 1, 12.5) == 10 / 0.0125
