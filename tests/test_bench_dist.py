"""Host logic of bench.py's multi-process path (replicas, one process per
GPU), on CPU ranks over gloo: the job time is the slowest rank's, the value
counts every rank's CSDs, and the reference arm runs on rank 0 only."""
import contextlib
import io
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    ms = bench.max_over_ranks(100.0 * (rank + 1), dist)
    value = bench.per_csd(ms, 2, ws)
    out = io.StringIO()
    if rank != 0:
        class A:  # the reference arm's arguments; ranks other than 0 do no work
            sample_n, n, steps, warmup, gpus = 8, 4096, 1, 0, ws
        with contextlib.redirect_stdout(out):
            bench.run_reference(A, rank, ws)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, ms, value, out.getvalue()))


def test_two_ranks_gloo():
    import torch.multiprocessing as mp
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value, printed in res:
        assert ms == 200.0                      # max over ranks
        assert value == pytest.approx(200.0 / 1e3 / (2 * ws))  # total CSDs = steps x ranks
        if rank != 0:
            assert printed == ""                # reference arm: rank 0 only


def test_single_process_helpers():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, None) == 12.5
    assert bench.per_csd(5000.0, 2, 1) == pytest.approx(2.5)
