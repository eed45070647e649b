"""The multi-GPU path runs independent replicas (transforms do not shard):
two gloo ranks on the CPU check the timing reduction bench.py uses."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    total, value = bench.aggregate_replicas(local_ms, steps=10, dist=dist, device="cpu")
    q.put((rank, total, value))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_timing_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, total, value in res:
        assert total == pytest.approx(200.0)              # max over ranks
        assert value == pytest.approx(2 * 10 / 0.2)       # all ranks' transforms / job time


def test_single_process_aggregate():
    import bench
    total, value = bench.aggregate_replicas(50.0, steps=5)
    assert total == 50.0 and value == pytest.approx(100.0)
