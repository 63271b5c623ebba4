"""The multi-rank logic of bench.py on CPU (gloo, world size 2): every rank
gets the slowest rank's time, the job value counts all ranks' rows, and the
reference arm runs on rank 0 only."""
import argparse
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank: int, ws: int, port: int, q) -> None:
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        t = bench._max_over_ranks(1.5 + rank, ws, torch.device("cpu"))
        q.put((rank, t, bench._job_rows_per_s(ws, 5, 1024, t)))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo_ws2():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, q), nprocs=2, join=True, start_method="spawn")
    got = sorted(q.get() for _ in range(2))
    assert [g[0] for g in got] == [0, 1]
    for _, t, v in got:
        assert t == 2.5                      # the slowest rank's time on every rank
        assert v == pytest.approx(2 * 5 * 1024 / 2.5)


def test_single_rank_is_identity():
    import bench
    assert bench._max_over_ranks(3.25, 1, None) == 3.25
    assert bench._job_rows_per_s(1, 4, 100, 2.0) == 200.0


def test_reference_arm_runs_on_rank0_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(workload="small_d256_l32", ref_rows=4, warmup=3, steps=2, gpus=2)
    bench.reference_arm(args)
    assert capsys.readouterr().out == ""
