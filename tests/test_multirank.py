"""The host side of the multi-GPU path, on CPU with two gloo ranks.

bench.py runs one process per GPU; every rank fuses and regularises its own street
(seed = rank) with no data-path collective, the job's time is the slowest rank's and
its work the sum over ranks.  These tests run that aggregation, the per-rank inputs
and the reference arm's rank gating as two processes on 127.0.0.1.
"""

import io
import os
import socket
import sys
from contextlib import redirect_stdout

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

torch = pytest.importorskip("torch")
mp = torch.multiprocessing


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    slowest = bench.max_over_ranks(10.0 * (rank + 1), world)
    total = bench.sum_over_ranks(100.0 * (rank + 1), world)
    # the reference arm runs on rank 0 only; the others return at once, printing nothing
    out = io.StringIO()
    if rank != 0:
        with redirect_stdout(out):
            bench.run_reference(None, rank, world)
    # each rank synthesises its own street
    _, d = bench.make_inputs(seed=rank, frames=range(1))
    q.put((rank, slowest, total, out.getvalue(), float(np.nansum(d))))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation_and_inputs():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in range(2):
        rank, slowest, total, printed, dsum = q.get(timeout=240)
        res[rank] = (slowest, total, printed, dsum)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == res[1][0] == 20.0  # max over ranks
    assert res[0][1] == res[1][1] == 300.0  # sum over ranks
    assert res[1][2] == ""  # rank 1 ran no reference and printed nothing
    assert res[0][3] != res[1][3]  # different streets per rank


def test_single_rank_helpers_are_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5 and bench.sum_over_ranks(7.0, 1) == 7.0
