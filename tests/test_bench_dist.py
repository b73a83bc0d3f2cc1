"""The benchmark's multi-rank bookkeeping on CPU: world_size-2 gloo ranks take
the slowest rank's time and count every rank's frames (weak scaling), and
non-zero ranks of the reference arm print nothing."""
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = [3.0, 5.0][rank]
    ms, value = bench.aggregate(7200, ms_local, world)
    bench.barrier(world)
    q.put((rank, ms, value))
    dist.destroy_process_group()


def test_aggregate_takes_slowest_rank_and_all_frames():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, ms, value in res:
        assert ms == pytest.approx(5.0)
        assert value == pytest.approx(2 * 7200 / 5e-3)


def test_reference_arm_non_zero_rank_is_silent(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench

    class A:
        steps, warmup, gpus = 1, 1, 2
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.reference_arm(A(), rank=1, world=2)
    assert buf.getvalue() == ""
    assert bench.aggregate(100, 4.0, 1) == (4.0, pytest.approx(25000.0))
