"""Host logic of the multi-GPU benchmark (independent replicas, one per GPU):
the slowest rank's time is taken and the job throughput counts every rank's
work. Run with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = bench.reduce_max(10.0 + 3.0 * rank, dist, "cpu")
    q.put((rank, ms, bench.job_throughput(world, 32, 20, ms)))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_and_job_throughput():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, thr in res:
        assert ms == 13.0                       # the slower rank
        assert thr == pytest.approx(2 * 32 * 20 / 0.013)


def test_single_process_identity():
    import bench
    assert bench.reduce_max(7.5, None, "cpu") == 7.5
    assert bench.job_throughput(1, 32, 10, 100.0) == pytest.approx(3200.0)
