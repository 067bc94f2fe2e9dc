"""Host logic of the benchmark's multi-GPU mode (independent replicas, one
per rank): the job time is the slowest rank's and the job throughput is the
sum over ranks -- checked with 2 gloo ranks on the CPU."""
import os
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        ms = bench.job_time_ms(100.0 + 50.0 * rank, ws, "cpu")
        q.put((rank, ms, bench.job_value(1e9, ws, ms)))
    finally:
        dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_the_work():
    import socket
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value in got:
        assert ms == 150.0                       # the slower rank's time on every rank
        assert value == pytest.approx(2 * 1e9 / 0.150)


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_time_ms(12.5, 1, "cpu") == 12.5
    assert bench.job_value(1e9, 1, 500.0) == pytest.approx(2e9)
