"""The multi-rank logic of bench.py on CPU (gloo, world size 2): every rank gets the largest
per-rank step time, the job value counts every rank's work, and the reference arm runs on
rank 0 only."""
import os
import sys

import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = [3.0, 5.0][rank]
    got = bench.max_over_ranks(ms, world, dist, "cpu")
    val = bench.job_value(1e9, got, world)
    dist.barrier()
    dist.destroy_process_group()

    class A:
        scale, steps, warmup = 10, 1, 0
    ref = bench.run_reference(A, rank, world) if rank == 1 else None   # non-zero ranks do no work
    q.put((rank, got, val, ref))


def test_max_over_ranks_and_job_value_gloo():
    import socket
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, got, val, ref in res:
        assert got == 5.0                              # the slowest rank's time, on every rank
        assert val == pytest.approx(2 * 1e9 / 5e-3 / 1e9)
    assert res[1][3] == 0                              # rank 1 of the reference arm exits at once


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(7.5, 1, None, "cpu") == 7.5
    assert bench.job_value(2e9, 2.0, 1) == pytest.approx(1000.0)
