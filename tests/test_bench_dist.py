"""bench.py's multi-rank plumbing with two gloo ranks on the CPU.

On a GPU node bench.py runs one process per GPU (torchrun), each solving an
independent problem; the ranks meet only at the barriers around the timed
region and in the max over ranks of its duration.  This runs that plumbing
with world size 2: process-group set-up from the torchrun environment, the
barrier, the max over ranks, and the reference arm doing its work on rank 0
only."""
import multiprocessing as mp
import os
import socket
import sys
import time

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class _Args:
    steps, warmup, gpus = 1, 0, 2


def _rank(rank, ws, port, q):
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(ws),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port),
                      CUDA_VISIBLE_DEVICES="")          # CPU ranks: bench picks gloo
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as td
    w, r, loc = bench.dist()
    assert td.get_backend() == "gloo"
    bench.barrier(w)
    t = bench.allmax(w, 0.25 * (rank + 1), "cpu")
    t0 = time.perf_counter()
    out = bench.reference_arm(_Args(), w, r) if r != 0 else None
    q.put((r, w, loc, t, out, time.perf_counter() - t0))
    bench.barrier(w)
    td.destroy_process_group()


def test_two_gloo_ranks_share_the_barrier_and_the_max_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [x[0] for x in res] == [0, 1]
    assert all(x[1] == 2 for x in res)
    assert [x[2] for x in res] == [0, 1]
    # every rank sees the slowest rank's time
    assert all(x[3] == pytest.approx(0.5) for x in res)
    # the reference arm does no work off rank 0
    assert res[1][4] is None and res[1][5] < 1.0
