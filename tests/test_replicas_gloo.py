"""The multi-GPU form of the benchmark runs independent replicas (one stream
per rank, no collective on the data path); ranks are joined only by the
max-over-ranks reduction of the step time. This checks that host logic with
two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank  # rank 1 is the slower replica
        m = bench.max_over_ranks(ms, world, "cpu")
        q.put((rank, m, bench.whole_job_gpoints(1000000, world, m)))
    finally:
        dist.destroy_process_group()


def test_two_replicas_report_all_pixels_over_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    for p in ps:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in got:
        assert m == 15.0  # both ranks see the slowest time
        assert v == pytest.approx(2 * 1000000 / 0.015 / 1e9)


def test_single_rank_needs_no_process_group():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1, "cpu") == 12.5
    assert bench.whole_job_gpoints(26214400, 1, 1.0) == pytest.approx(26.2144)
