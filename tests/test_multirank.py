"""The N > 1 path of bench.py (replicas; no data-path collective): the whole-job value is all
ranks' points over the slowest rank's time, identical on every rank.  Two gloo ranks on CPU."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = [1000.0, 1600.0][rank]          # rank 1 is the slow one
    value, ms_max = bench.job_value(64, 5, ms_local)
    out[rank] = (value, ms_max)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_rank():
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    expect = 64 * 5 * 2 / 1.6
    for r in range(2):
        value, ms_max = out[r]
        assert ms_max == 1600.0
        assert value == pytest.approx(expect)


def test_single_process_value():
    import bench
    value, ms_max = bench.job_value(64, 5, 2000.0)
    assert ms_max == 2000.0 and value == pytest.approx(160.0)
