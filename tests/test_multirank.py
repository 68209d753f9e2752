"""Multi-rank host logic of the benchmark on CPU: two gloo ranks, each with its
own independent stream of solves, aggregate to the whole-job rate (units of all
ranks over the slowest rank's time)."""

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

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    units = [30.0, 50.0][rank]
    elapsed = [2.0, 4.0][rank]
    rate = bench.job_throughput(dist, units, elapsed, device="cpu")
    mx = bench.max_over_ranks(dist, elapsed, device="cpu")
    out[rank] = (rate, mx)
    dist.destroy_process_group()


def test_job_throughput_over_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        rate, mx = out[r]
        assert mx == 4.0
        assert rate == pytest.approx(80.0 / 4.0)


def test_single_process_is_identity():
    import bench

    assert bench.job_throughput(None, 12.0, 3.0) == 4.0
