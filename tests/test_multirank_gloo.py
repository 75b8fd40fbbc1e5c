"""The multi-rank path of bench.py on CPU: two gloo ranks, each timing its
own job (weak scaling, no data-path collective); the job rate is all ranks'
units over the slowest rank's time."""
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


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [10.0, 25.0][rank]
    units_local = [1000, 3000][rank]
    ms, value = bench.aggregate(ms_local, units_local, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_rank_weak_scaling_aggregate():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(2):
        ms, value = out[r]
        assert ms == pytest.approx(25.0)
        assert value == pytest.approx(4000 / 0.025)


def test_single_rank_aggregate():
    import bench
    ms, value = bench.aggregate(20.0, 500)
    assert ms == 20.0 and value == pytest.approx(25000.0)
