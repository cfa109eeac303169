"""The multi-rank bookkeeping of bench.py on CPU (gloo, world size 2).

With N ranks every rank advances its own grid (independent replicas, weak scaling); the only
exchange is the barrier and the max over ranks of the timed region, from which the whole-job value
is computed.  The reference arm runs on rank 0 alone.
"""
import argparse
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        m = bench.reduce_max(times[rank], world, "cpu")
        v = bench.job_value(world, 4096 * 4096, 20, m)
        q.put((rank, m, v))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_both_grids():
    world, times = 2, [0.75, 1.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, times, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, m, v in out:
        assert m == max(times)
        assert v == pytest.approx(world * 4096 * 4096 * 20 / max(times))


def test_single_rank_is_identity():
    import bench
    assert bench.reduce_max(0.5, 1, "cpu") == 0.5
    assert bench.job_value(1, 10, 3, 2.0) == 15.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    from paper_1206_3229_gb300 import inputs as I
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(steps=5, warmup=3, gpus=2)
    assert bench.run_reference(args, I.HMF_256) == 0
    assert capsys.readouterr().out == ""
