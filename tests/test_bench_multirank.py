"""bench.py's multi-rank path on the CPU: two gloo ranks, each timing its own replica, reduce to the
whole-job rate (units of all ranks over the slowest rank's time) with no data-path collective."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup("gloo")
    assert (w, r, local) == (ws, rank, rank)
    bench.barrier(w)
    # rank r processed (r + 1) * 1000 units in (r + 1) seconds
    rate, sec, units = bench.job_rate((rank + 1) * 1000.0, float(rank + 1), w)
    q.put((rank, rate, sec, units))
    dist.destroy_process_group()


def test_two_rank_job_rate():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, rate, sec, units in res:
        assert sec == 2.0 and units == 3000.0 and rate == pytest.approx(1500.0)


def test_single_rank_needs_no_process_group(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.dist_setup("gloo") == (1, 0, 0)
    assert bench.job_rate(10.0, 2.0, 1) == (5.0, 2.0, 10.0)
