"""Multi-rank host logic of bench.py on CPU: two gloo ranks, whole-job throughput
= units summed over ranks / max time over ranks."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units, secs = bench.aggregate(local_units=3 + rank, local_seconds=1.0 + 0.5 * rank)
    out[rank] = (units, secs)
    dist.barrier()
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    ctx = mp.get_context("spawn")
    world = 2
    port = _free_port()
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    for r in range(world):
        assert res[r] == pytest.approx((7.0, 1.5))


def test_aggregate_single_process_is_identity():
    import bench
    assert bench.aggregate(5, 2.0) == (5, 2.0)
