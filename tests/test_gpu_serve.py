"""Serving loop (spmv_server_*) through the C ABI.

* Every result is the same alone and in the mix: each request is first run alone (one slot,
  batches of one, submitted and awaited one at a time), then all of them are replayed
  arriving together on four slots (so SpMV requests are batched and slots overlap); the
  two sets of results must be bitwise equal, and equal to spmv_mul / spmv_pagerank.
* SpMV results also match the oracle (FP64 within 1e-13 (|A||x|); FP32 within the FP32
  accumulation bound), PageRank results the oracle's iteration.
* Admission by memory: with a budget that holds the resident set and one request, the
  server defers admissions and never exceeds the budget; a request that cannot fit at all
  fails with SPMV_ERR_OOM.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


def make_mats(sp, f32=False):
    out = []
    for i, scale in enumerate([10, 12, 13, 11]):
        n = 1 << scale
        r, c = synth.rmat(scale, 16, seed=200 + i)
        v = synth.values(r, c, 300 + i)
        if f32:
            v = v.astype(np.float32).astype(np.float64)
        vd = torch.from_numpy(v.astype(np.float32) if f32 else v).to(DEV)
        h = sp.spmv_create_coo(n, n, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV), vd)
        sp.spmv_convert(h, "merge" if i % 2 == 0 else "rowsplit")
        rp, co, vo = oracle.coo_to_csr(n, n, r, c, v)
        out.append((h, n, rp, co, vo))
    return out


def build_requests(sp, mats, dt, nreq=24, seed=0):
    """A mix of SpMV (three accumulations for FP32 vectors) and PageRank requests with
    pinned host inputs and outputs."""
    rng = np.random.Generator(np.random.PCG64(seed))
    reqs, keep = [], []
    for q in range(nreq):
        mi = int(rng.integers(0, len(mats)))
        h, n, *_ = mats[mi]
        if q % 5 == 4:
            y = torch.empty(n, dtype=torch.float64).pin_memory()
            reqs.append(("pr", mi, None, y, 20 if q % 2 else 7))
        else:
            x = torch.from_numpy(synth.vector(n, 1000 + q).astype(dt)).pin_memory()
            y = torch.full((n,), float("nan"), dtype=torch.float64 if dt == np.float64 else torch.float32).pin_memory()
            acc = [sp.SPMV_ACC_DEFAULT, sp.SPMV_ACC_COMPENSATED, sp.SPMV_ACC_F64][q % 3] if dt == np.float32 else sp.SPMV_ACC_F64
            reqs.append(("spmv", mi, x, y, acc))
    return reqs


def to_struct(sp, ids, rq):
    kind, mi, x, y, extra = rq
    if kind == "pr":
        return sp.Server.request(sp.SPMV_REQ_PAGERANK, ids[mi], y, iters=extra, damping=0.85)
    return sp.Server.request(sp.SPMV_REQ_SPMV, ids[mi], y, x=x, accum=extra)


@pytest.mark.parametrize("f32", [False, True])
def test_same_alone_and_in_mix(sp, f32):
    dt = np.float32 if f32 else np.float64
    mats = make_mats(sp, f32=f32)
    reqs = build_requests(sp, mats, dt, seed=int(f32))
    budget = 4 << 30
    # alone: one slot, batches of one, one request at a time
    solo = sp.Server(budget, slots=1, max_batch=1)
    ids = [solo.add(m[0]) for m in mats]
    alone = []
    for rq in reqs:
        t = solo.submit(to_struct(sp, ids, rq))
        assert solo.wait(t) > 0
        alone.append(rq[3].numpy().copy())
        rq[3].fill_(float("nan"))
    solo.close()
    # in the mix: everything arrives together on four slots
    srv = sp.Server(budget, slots=4, max_batch=16)
    ids = [srv.add(m[0]) for m in mats]
    lat = srv.replay([to_struct(sp, ids, rq) for rq in reqs], np.zeros(len(reqs)))
    st = srv.stats()
    srv.close()
    assert (lat > 0).all() and st["completed"] == len(reqs) and st["failed"] == 0
    assert st["batched_requests"] > st["launches"]          # some SpMV requests shared a launch
    for rq, a in zip(reqs, alone):
        assert np.array_equal(rq[3].numpy(), a, equal_nan=False), rq[:2]
    # against the direct calls and the oracle
    u = 2.0 ** -24
    for rq, a in zip(reqs, alone):
        kind, mi, x, y, extra = rq
        h, n, rp, co, vo = mats[mi]
        if kind == "pr":
            xd = torch.empty(n, dtype=torch.float64, device=DEV)
            sp.spmv_pagerank(h, xd, 0.85, extra)
            torch.cuda.synchronize()
            assert np.array_equal(xd.cpu().numpy(), a)
            ref = oracle.pagerank(rp, co, 0.85, extra)
            assert np.abs(a - ref).max() <= 1e-12
            continue
        xd = x.to(DEV)
        yd = torch.empty(n, dtype=xd.dtype, device=DEV)
        sp.spmv_convert(h, "merge")
        sp.spmv_mul(h, xd, yd, accum=extra)
        torch.cuda.synchronize()
        assert np.array_equal(yd.cpu().numpy(), a), (mi, extra)
        x64 = x.numpy().astype(np.float64)
        ref = oracle.csr_spmv(rp, co, vo, x64)
        scale = oracle.csr_absmul(rp, co, vo, x64)
        if not f32:
            assert (np.abs(a - ref) <= 1e-13 * scale).all()
        else:
            L = np.diff(rp).astype(np.float64)
            g = (L + 1) * u / (1 - (L + 1) * u)
            assert (np.abs(a.astype(np.float64) - ref) <= g * scale + u * np.abs(ref)).all()
    for m in mats:
        sp.spmv_destroy(m[0])


def test_admission_by_memory(sp):
    mats = make_mats(sp)
    srv0 = sp.Server(8 << 30, slots=1, max_batch=1)
    for m in mats:
        srv0.add(m[0])
    resident = srv0.stats()["resident_bytes"]
    srv0.close()
    # room for the resident set and about 1.5 requests of the largest matrix (x, y and the
    # batch scratch of 20 bytes per tile)
    n_max = max(m[1] for m in mats)
    tiles_max = max(sp.spmv_info(m[0])["merge_tiles"] for m in mats)
    budget = resident + int(1.5 * (2 * n_max * 8 + tiles_max * 20 + 4096))
    srv = sp.Server(budget, slots=4, max_batch=16)
    ids = [srv.add(m[0]) for m in mats]
    reqs = [rq for rq in build_requests(sp, mats, np.float64, nreq=16, seed=5) if rq[0] == "spmv"]
    lat = srv.replay([to_struct(sp, ids, rq) for rq in reqs], np.zeros(len(reqs)))
    st = srv.stats()
    assert (lat > 0).all() and st["completed"] == len(reqs)
    assert st["peak_bytes"] <= budget and st["deferred"] > 0
    for rq in reqs:
        h, n, rp, co, vo = mats[rq[1]]
        x64 = rq[2].numpy()
        ref = oracle.csr_spmv(rp, co, vo, x64)
        assert (np.abs(rq[3].numpy() - ref) <= 1e-13 * oracle.csr_absmul(rp, co, vo, x64)).all()
    srv.close()
    # a request that cannot fit even alone fails instead of waiting forever
    tight = sp.Server(resident + 1024, slots=2, max_batch=4)
    ids = [tight.add(m[0]) for m in mats]
    h, n, *_ = mats[2]
    x = torch.zeros(n, dtype=torch.float64).pin_memory()
    y = torch.zeros(n, dtype=torch.float64).pin_memory()
    t = tight.submit(sp.Server.request(sp.SPMV_REQ_SPMV, ids[2], y, x=x))
    with pytest.raises(sp.SpmvError) as e:
        tight.wait(t)
    assert e.value.status == sp.SPMV_ERR_OOM
    tight.close()
    for m in mats:
        sp.spmv_destroy(m[0])


def test_poisson_replay_reports_latencies(sp):
    mats = make_mats(sp, f32=True)
    srv = sp.Server(4 << 30, slots=4, max_batch=32)
    ids = [srv.add(m[0]) for m in mats]
    kind, mat = synth.request_mix(300, len(mats), 0.2, seed=9)
    arrivals = synth.poisson_arrivals(5000.0, 300, seed=9)
    bufs, reqs = [], []
    for k, mi in zip(kind, mat):
        n = mats[mi][1]
        if k == 1:
            y = torch.empty(n, dtype=torch.float64).pin_memory()
            reqs.append(sp.Server.request(sp.SPMV_REQ_PAGERANK, ids[mi], y, iters=20))
        else:
            x = torch.from_numpy(synth.vector(n, 7).astype(np.float32)).pin_memory()
            y = torch.empty(n, dtype=torch.float32).pin_memory()
            reqs.append(sp.Server.request(sp.SPMV_REQ_SPMV, ids[mi], y, x=x))
            bufs.append(x)
        bufs.append(y)
    lat = srv.replay(reqs, arrivals)
    st = srv.stats()
    srv.close()
    assert (lat > 0).all() and st["completed"] == 300
    p50, p99 = np.percentile(lat, [50, 99])
    assert 0 < p50 <= p99 < 5.0
    for m in mats:
        sp.spmv_destroy(m[0])
