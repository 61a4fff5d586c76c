"""bench.py's multi-rank aggregation on CPU: two gloo ranks (no GPU).  Every rank times its own
replica of the workload; the job's time is the slowest rank's, and its rate counts every rank's
pixels over that time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms = [0.25, 0.40][rank]
    got = bench.max_over_ranks(ms, world, torch.device("cpu"))
    q.put((rank, got, bench.job_rate(8192 * 8192, world, got)))
    dist.destroy_process_group()


def test_max_over_ranks_and_job_rate_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, got, rate in res:
        assert got == pytest.approx(0.40)
        assert rate == pytest.approx(2 * 8192 * 8192 / 0.40e-3 / 1e9)


def test_single_rank_passthrough():
    import bench
    assert bench.max_over_ranks(0.3, 1, torch.device("cpu")) == 0.3
    assert bench.job_rate(100, 1, 1.0) == pytest.approx(100 / 1e-3 / 1e9)
