"""The benchmark's multi-rank host logic on CPU with the gloo backend (world size 2).

Elements are independent, so N ranks each integrate their own copy of the workload
(weak scaling) with no collective in the data path; the only cross-rank steps are the
barriers and the max-over-ranks step time.  These tests run that reduction on two gloo
ranks, check the whole-job rate built from it, and check that the reference arm does its
work on rank 0 only.
"""
import argparse
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, times, results):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        t = bench.max_over_ranks(times[rank], world)
        results[rank] = (t, bench.job_throughput(world, 4096, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_gloo():
    world = 2
    times = [0.0031, 0.0047]               # seconds per step on each rank
    with mp.get_context("spawn").Manager() as m:       # no fork of a multi-threaded process
        results = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), times, results), nprocs=world, join=True)
        got = dict(results)
    for r in range(world):
        t, v = got[r]
        assert t == max(times)
        assert v == pytest.approx(world * 4096 / max(times))


def test_single_rank_is_identity():
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.job_throughput(1, 4096, 0.5) == 8192.0


def test_reference_arm_rank_nonzero_does_nothing(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(warmup=3, steps=5, gpus=2)
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.run_reference(args)            # returns before touching the oracle
    assert buf.getvalue() == ""
