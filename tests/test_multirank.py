"""Replica path of bench.py on CPU: two gloo ranks (world size 2) take the max of their times over
the ranks, meet at the barrier, and report the whole-job value of independent replicas."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import sys
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bench._WORLD[0] = world
    bench.barrier()
    t = bench.max_over_ranks(10.0 + 5.0 * rank)  # rank 1 is the slow one
    out[rank] = (t, bench.replica_value(world, 1000, 4, t))
    bench.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_replica_value():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        codes = [p.exitcode for p in procs]
        res = dict(out)
    assert codes == [0, 0], codes
    for r in range(world):
        t, v = res[r]
        assert t == 15.0
        assert v == pytest.approx(2 * 1000 * 4 / 15e-3)


def test_single_rank_is_the_identity():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    bench._WORLD[0] = 1
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.replica_value(1, 100, 2, 4.0) == pytest.approx(100 * 2 / 4e-3)
