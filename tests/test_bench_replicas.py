"""bench.py's multi-rank timing (replicas, no data-path collective): the
slowest rank's time and the whole-job rate, over world_size 2 on CPU (gloo)."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        secs = 2.0 + rank          # rank 1 is the slow one
        t, rate = bench.job_rate(100.0, secs, dist, "cpu")
        dist.barrier()
        out.put((rank, t, rate))
    finally:
        dist.destroy_process_group()


def test_job_rate_takes_the_slowest_rank_and_all_units():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, rate in res:
        assert t == 3.0                    # max over ranks
        assert rate == 100.0 * 2 / 3.0     # units of both ranks / slowest time


def test_job_rate_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.job_rate(50.0, 2.0) == (2.0, 25.0)
