"""The multi-process side of bench.py, on CPU with the gloo backend and two ranks: timings are
combined as the maximum over ranks (the job is as slow as its slowest replica), the whole-job
rate of N replicas is N times one replica's, and the reference arm prints only on rank 0."""
import contextlib
import io
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks([1.0 + rank, 10.0 - rank, 3.0])
        buf = io.StringIO()

        class Args:
            steps, warmup, gpus = 1, 0, world
        if rank != 0:  # the reference arm does no work and prints nothing off rank 0
            with contextlib.redirect_stdout(buf):
                bench.run_reference(Args, rank, world)
        out[rank] = (got, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_rank_timing_and_reference_arm():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    for r in range(world):
        got, printed = out[r]
        assert got == [2.0, 10.0, 3.0]
    assert out[1][1] == ""
    assert bench.replicas_value(2.0, 2) == 2 * bench.replicas_value(2.0, 1) == 1000.0
    assert bench.max_over_ranks([4.0, 5.0]) == [4.0, 5.0]  # single process
