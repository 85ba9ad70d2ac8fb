"""bench.py's multi-GPU path runs independent replicas (the solver does not
shard): the job value is all ranks' work over the slowest rank's time.  The
host logic is checked here with two gloo ranks on the CPU."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local = 100.0 + 50.0 * rank
        mx = bench.max_over_ranks(local)
        out[rank] = (mx, bench.job_value(1000, 4, world, mx))
    finally:
        dist.destroy_process_group()


def test_two_replicas_max_time_and_job_value():
    world = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0] == res[1]
    mx, val = res[0]
    assert mx == 150.0
    assert val == pytest.approx(2 * 1000 * 4 / 0.150)


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5) == 12.5
    assert bench.job_value(10, 2, 1, 1000.0) == pytest.approx(20.0)
