"""The N > 1 path of bench.py on CPU: world size 2 over gloo.

Each rank is a replica solving its own problem; the job time is the slowest
rank's (all_reduce MAX), the job throughput counts every rank's DOF, and the
reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys
import types

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, times, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        assert bench._dist() == (ws, rank, rank)
        ms = bench.max_over_ranks(dist, times[rank], "cpu")
        value = bench.job_throughput(ws, 1e8, ms)
        buf = io.StringIO()
        if rank != 0:
            # the reference arm is rank 0's alone: other ranks return at once, silently
            with contextlib.redirect_stdout(buf):
                bench.run_reference(types.SimpleNamespace(steps=1, warmup=3, gpus=ws))
        dist.barrier()
        out[rank] = (ms, value, buf.getvalue())
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_gloo():
    ws = 2
    times = [120.0, 135.5]
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(ws, _free_port(), times, out), nprocs=ws, join=True,
                           start_method="spawn")
        res = dict(out)
    for rank in range(ws):
        ms, value, printed = res[rank]
        assert ms == max(times)
        assert value == pytest.approx(ws * 1e8 / (max(times) * 1e-3), rel=1e-15)
    assert res[1][2] == ""


def test_single_rank_is_identity():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, 3.25, "cpu") == 3.25
    assert bench.job_throughput(1, 1e8, 100.0) == pytest.approx(1e9)
