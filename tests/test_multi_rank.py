"""The row-partitioned multi-GPU product's host logic on CPU: two gloo ranks, each multiplies its
row range (the oracle stands in for the rank's GPU product) and the all-gathered y equals the
single-rank product bit for bit; the cut points are the merge-path split of Section 3.3 at rank
granularity (checked against the oracle's merge-path search)."""
import os
import sys

import numpy as np
import pytest

from conftest import ROOT

torch = pytest.importorskip("torch")


def _rank(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_2502_19284_gb300 import partition
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    n = 1 << 12
    r, c = synth.rmat(12, 16, seed=9)
    v = synth.values(r, c, 9)
    x = synth.vector(n, 10)
    rp, co, vo = oracle.coo_to_csr(n, n, r, c, v)
    cuts = partition.row_ranges(rp, world)
    lrp, lco, lvo = partition.local_rows(rp, co, vo, int(cuts[rank]), int(cuts[rank + 1]))
    y_local = oracle.csr_spmv(lrp, lco, lvo, x)
    y = partition.gather_y(dist, y_local, cuts)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, cuts.tolist(), y.tobytes()))


def test_row_partitioned_product_two_gloo_ranks():
    import socket
    import torch.multiprocessing as mp
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=180) for _ in range(2))   # drain the queue before joining
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    n = 1 << 12
    r, c = synth.rmat(12, 16, seed=9)
    v = synth.values(r, c, 9)
    x = synth.vector(n, 10)
    rp, co, vo = oracle.coo_to_csr(n, n, r, c, v)
    want = oracle.csr_spmv(rp, co, vo, x)
    for rank, cuts, yb in res:
        assert np.array_equal(np.frombuffer(yb, dtype=np.float64), want)   # every rank holds all of y
        assert cuts == res[0][1]


@pytest.mark.parametrize("parts", [1, 2, 3, 8])
def test_row_ranges_are_the_merge_path_split(parts):
    """Cut g is the row count consumed at diagonal g (m + nnz) / parts of the merge path."""
    sys.path.insert(0, ROOT)
    import oracle
    import synth
    from paper_2502_19284_gb300 import partition
    rows, cols = synth.rmat(10, 16, seed=4)
    rp, _, _ = oracle.coo_to_csr(1 << 10, 1 << 10, rows, cols, None)
    m, nnz = rp.size - 1, int(rp[-1])
    cuts = partition.row_ranges(rp, parts)
    assert cuts[0] == 0 and cuts[-1] == m and (np.diff(cuts) >= 0).all()
    for g in range(1, parts):
        d = g * (m + nnz) // parts
        assert cuts[g] == oracle.merge_path_search(d, rp)[0]
        # balance: rows plus nonzeros of every part within one row of the mean
    sizes = [(cuts[g + 1] - cuts[g]) + (rp[cuts[g + 1]] - rp[cuts[g]]) for g in range(parts)]
    assert max(sizes) - min(sizes) <= 2 + int(np.diff(rp).max())
