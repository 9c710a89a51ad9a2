"""The N > 1 path of bench.py on CPU: independent replicas, one per rank,
joined only by the timing reduction (max over ranks) and the whole-job rate.
Two gloo ranks in spawned processes."""
import socket

import pytest
import torch.multiprocessing as mp

import bench

from rank_worker import replica_rank


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def test_two_replicas_report_the_slowest_rank_and_the_whole_job():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=replica_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        res = sorted(q.get(timeout=120) for _ in range(2))
    finally:
        for p in procs:
            p.join(timeout=60)
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, ms, rate in res:
        assert ms == 11.0  # every rank sees the slowest replica's time
        assert rate == pytest.approx(2 * 200 * 50 / 0.011)


def test_single_process_keeps_its_own_time():
    assert bench.slowest_rank(7.5, "cpu") == 7.5
    assert bench.whole_job_rate(1, 200, 10, 0.5) == 4000.0
