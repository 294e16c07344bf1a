"""The multi-GPU path is independent replicas (the PM solve does not shard):
check the whole-job aggregation of bench.py with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import bench

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "took" 2 + r seconds for 5 evaluations
    value, slowest = bench.replica_throughput(2.0 + rank, 5, world, "cpu")
    out[rank] = (value, slowest)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_replica_throughput_two_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(100)
            assert p.exitcode == 0
        res = dict(out)
    # slowest rank bounds the job; all ranks agree; value counts all ranks' work
    for r in range(world):
        value, slowest = res[r]
        assert slowest == pytest.approx(3.0)
        assert value == pytest.approx(world * 5 / 3.0)
