"""The multi-rank path of bench.py on CPU: two gloo ranks in separate processes.

Under torchrun every rank runs its own reconstructions (weak scaling, no
collective on the data path); the only exchange is the all-reduce MAX of the
ranks' times, and the whole-job value counts every rank's reconstructions over
the slowest rank's time.  The reference arm runs on rank 0 only.
"""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [120.0, 250.0][rank]  # the second rank is the slower one
        m = bench.max_over_ranks(local_ms, dist, "cpu")
        q.put((rank, m, bench.job_value(world, 5, m)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_report_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, m, v in got:
        assert m == 250.0, (rank, m)
        assert v == pytest.approx(2 * 5 / 0.25)  # 10 reconstructions in the slowest rank's 0.25 s


def test_single_process_value():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(40.0) == 40.0
    assert bench.job_value(1, 4, 40.0) == pytest.approx(100.0)


def test_reference_arm_other_ranks_do_nothing(capsys):
    sys.path.insert(0, ROOT)
    import argparse

    import bench

    args = argparse.Namespace(steps=1, warmup=0, gpus=2)
    assert bench.reference_arm(args, rank=1) is None
    assert capsys.readouterr().out == ""
