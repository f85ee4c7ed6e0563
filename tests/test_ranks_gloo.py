"""The multi-rank bookkeeping of bench.py on CPU with two gloo ranks: every
rank learns the slowest rank's time, and the job throughput counts all
replicas over that time (replicas only: the data path has no collective)."""
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


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = 10.0 + 5.0 * rank  # rank 1 is slower
    ms = bench.max_over_ranks(local_ms, dist, device="cpu")
    value = bench.job_mlups(world, 1000, 4, ms)
    q.put((rank, ms, value))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_max_time_and_job_throughput():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in res:
        assert ms == 15.0
        assert abs(value - 2 * 1000 * 4 / 15e-3 / 1e6) < 1e-9


def test_single_process_is_the_identity():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
    assert abs(bench.job_mlups(1, 2_000_000, 10, 20.0) - 1000.0) < 1e-9
