"""The multi-rank path of bench.py on CPU ranks (gloo, world size 2): the step
time is the maximum over ranks and the rate counts every rank's queries."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = [12.5, 30.25][rank]
    job = bench.max_over_ranks(ms, "cpu")
    out[rank] = (job, bench.whole_job_rate(3597, 5, world, job))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][0] == out[1][0] == 30.25
    assert out[0][1] == pytest.approx(3597 * 5 * 2 / 0.03025)


def test_single_process_is_unchanged():
    import bench

    assert bench.max_over_ranks(7.0) == 7.0
    assert bench.whole_job_rate(100, 2, 1, 1000.0) == 200.0
