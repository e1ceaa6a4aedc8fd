"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas), the
reported time is the slowest rank's, and the job rate counts every replica."""
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
    ms = 100.0 + 50.0 * rank  # rank 1 is the slow one
    mx = bench.max_over_ranks(ms, dist, "cpu")
    out[rank] = (mx, bench.job_rate(10, mx, world))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_report_max_and_job_rate():
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
    assert out[0] == out[1]
    mx, rate = out[0]
    assert mx == 150.0
    assert rate == pytest.approx(2 * 10 / 0.150)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.job_rate(5, 100.0, 1) == pytest.approx(50.0)
