"""The multi-rank bench path on CPU: two gloo ranks, each timing its own replica;
the job's time is the slowest rank's and its throughput counts every rank's cells."""
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


def _rank(rank, world, port, q):
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [120.0, 150.0][rank]
    q.put((rank, bench.aggregate(ms_local, 1000, 10, world, dist, "cpu")))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_and_sum_the_cells():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = got[r]
        assert ms == 150.0
        assert value == pytest.approx(1000 * 10 * 2 / 0.150)


def test_single_rank_aggregate():
    import bench
    ms, value = bench.aggregate(50.0, 100, 4, 1)
    assert ms == 50.0 and value == pytest.approx(100 * 4 / 0.05)
