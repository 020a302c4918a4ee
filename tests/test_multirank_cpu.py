"""The multi-GPU path of bench.py (one process per GPU, independent replicas)
exercised on the host: two gloo ranks agree on the job time (the slowest
rank's), count every rank's pixels in the job rate and solve different
problems.  No GPU: the reductions run on CPU tensors."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        local_ms = 10.0 + 5.0 * rank            # the ranks' own timed regions
        job_ms = bench.max_over_ranks(local_ms, world)
        rate = bench.job_throughput(1000, world, 4, job_ms)
        cfg = dict(bench.WORKLOADS["denoise4096"], h=16, w=16)
        y = bench._problem(cfg, rank).y
        out.put((rank, job_ms, rate, bench.replica_seed(cfg["seed"], rank), float(y.sum())))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_job_time_and_rate():
    mp = pytest.importorskip("torch.multiprocessing")
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, t0, v0, s0, y0), (_, t1, v1, s1, y1) = res
    assert t0 == t1 == 15.0                      # slowest rank
    assert v0 == v1 == pytest.approx(1000 * 2 * 4 / 0.015 / 1e6)
    assert s0 != s1 and y0 != y1                 # independent replicas
