"""The N > 1 path of bench.py on CPU: two gloo ranks aggregate whole-job units
(sum over ranks) and times (max over ranks) as the GPU replicas do."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, times = bench.aggregate_ranks([1000.0 * (rank + 1), float(rank)], [0.5 + rank, 2.0 - rank])
    q.put((rank, units, times))
    dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    import torch.multiprocessing as mp
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
    for rank, units, times in out:
        assert units == [3000.0, 1.0]     # sum over ranks
        assert times == [1.5, 2.0]        # max over ranks


def test_single_process_passthrough():
    import bench
    assert bench.aggregate_ranks([5.0], [2.0]) == ([5.0], [2.0])
