"""The multi-GPU path of bench.py runs independent replicas (one per rank) and combines
them only through the rank aggregation: max of the timed seconds, sum of the crossings.
Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    t, c = bench.aggregate_ranks(1.0 + rank, 1000 * (rank + 1))
    q.put((rank, t, c))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, c in out:
        assert t == 2.0 and c == 3000.0


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_ranks(0.5, 7) == (0.5, 7.0)
