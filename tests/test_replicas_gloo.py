"""The N > 1 bench path: independent replicas, max-over-ranks time, summed work
(world size 2, gloo on CPU; no collective on the data path)."""
import multiprocessing as mp
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 1000.0 * (rank + 1)             # rank 1 is the slow one
    ms, value = bench.aggregate(ms_local, units_per_rank=2048, dist=dist, device="cpu")
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_replicas_take_max_time_and_sum_work():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 2000.0                    # max over ranks
        assert value == pytest.approx(2 * 2048 / 2.0)


def test_single_rank_aggregate():
    import bench
    ms, value = bench.aggregate(500.0, 1000)
    assert ms == 500.0 and value == pytest.approx(2000.0)
