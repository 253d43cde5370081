"""Batched multi-RHS products spmv_mul_batch (Y_i = A_i X_i, k = 1..16 right-hand sides)
through the C ABI.

Checks, on seeded R-MAT / Zipf / Erdos-Renyi matrices of mixed sizes in one batch:
  * against the oracle's multiple-vector product within |Y - Yref| <= 1e-13 (|A||X|)
    (FP64), and bit-exact on integer data;
  * per column, bitwise equal to spmv_mul on the merge path with the same accumulation
    (the batch walks the same tiles in the same order);
  * graph replay with new X / Y, on-demand merge tiles for handles in other formats,
    empty matrices, and argument errors.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-13


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


def patterns():
    r, c = synth.rmat(13, 16, seed=71)
    yield 1 << 13, 1 << 13, r, c
    r, c = synth.zipf_rows(3000, 1.8, 2500, 0.1, seed=72)
    perm = synth.shuffle_order(r.size, 4)
    yield 3000, 3000, r[perm], c[perm]
    r, c = synth.erdos_renyi(777, 5, seed=73)
    yield 777, 777, r, c
    yield 50, 40, np.zeros(0, np.int32), np.zeros(0, np.int32)   # all rows empty


def build(sp, integer=False, kind="f64", fmt="merge"):
    mats = []
    for i, (m, n, r, c) in enumerate(patterns()):
        v = synth.values(r, c, 80 + i, integer=integer)
        if kind == "f32":
            v = v.astype(np.float32).astype(np.float64)
            vd = torch.from_numpy(v.astype(np.float32)).to(DEV)
        elif kind == "pattern":
            v = np.ones(r.size)
            vd = None
        else:
            vd = torch.from_numpy(v).to(DEV)
        h = sp.spmv_create_coo(m, n, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV), vd,
                               dtype=sp.SPMV_PATTERN if kind == "pattern" else None)
        sp.spmv_convert(h, fmt)
        rp, co, vo = oracle.coo_to_csr(m, n, r, c, v)
        mats.append((h, m, n, rp, co, vo))
    return mats


def rhs(n, k, seed, integer=False, dtype=np.float64):
    X = np.stack([synth.vector(n, seed + q, integer=integer) for q in range(k)], axis=1) if n else np.zeros((0, k))
    return np.ascontiguousarray(X.astype(dtype))


@pytest.mark.parametrize("k", [1, 3, 4, 8, 16])
def test_batch_f64_against_oracle_and_single(sp, k):
    mats = build(sp)
    Xs = [rhs(n, k, 100 * k + i) for i, (_, m, n, *_r) in enumerate(mats)]
    Xd = [torch.from_numpy(X).to(DEV) for X in Xs]
    Yd = [torch.full((m, k), float("nan"), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
    sp.spmv_mul_batch([t[0] for t in mats], Xd, Yd, k=k)
    torch.cuda.synchronize()
    for (h, m, n, rp, co, vo), X, Xt, Yt in zip(mats, Xs, Xd, Yd):
        Y = Yt.cpu().numpy()
        ref = oracle.csr_spmm(rp, co, vo, X)
        for q in range(k):
            scale = oracle.csr_absmul(rp, co, vo, X[:, q])
            assert (np.abs(Y[:, q] - ref[:, q]) <= TOL * scale).all(), (m, q)
            y1 = torch.empty(m, dtype=torch.float64, device=DEV)
            sp.spmv_mul(h, Xt[:, q].contiguous(), y1, accum=sp.SPMV_ACC_F64)
            torch.cuda.synchronize()
            assert np.array_equal(Y[:, q], y1.cpu().numpy()), (m, q)
    for t in mats:
        sp.spmv_destroy(t[0])


def test_batch_integer_exact(sp):
    k = 8
    mats = build(sp, integer=True)
    Xs = [rhs(n, k, 7 + i, integer=True) for i, (_, m, n, *_r) in enumerate(mats)]
    Yd = [torch.empty((m, k), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
    sp.spmv_mul_batch([t[0] for t in mats], [torch.from_numpy(X).to(DEV) for X in Xs], Yd, k=k)
    torch.cuda.synchronize()
    for (h, m, n, rp, co, vo), X, Yt in zip(mats, Xs, Yd):
        assert np.array_equal(Yt.cpu().numpy(), oracle.csr_spmm(rp, co, vo, X))
        sp.spmv_destroy(h)


@pytest.mark.parametrize("kind,acc", [("f32", "F32"), ("f32", "COMPENSATED"), ("f32", "SEGMENT"), ("f32", "F64"),
                                      ("pattern", "F32"), ("pattern", "COMPENSATED"), ("pattern", "SEGMENT")])
def test_batch_f32_bitwise_equal_to_single(sp, kind, acc):
    k = 4
    accv = getattr(sp, "SPMV_ACC_" + acc)
    mats = build(sp, kind=kind)
    Xs = [rhs(n, k, 300 + i, dtype=np.float32) for i, (_, m, n, *_r) in enumerate(mats)]
    Xd = [torch.from_numpy(X).to(DEV) for X in Xs]
    Yd = [torch.full((m, k), float("nan"), dtype=torch.float32, device=DEV) for (_, m, *_r) in mats]
    sp.spmv_mul_batch([t[0] for t in mats], Xd, Yd, k=k, accum=accv)
    torch.cuda.synchronize()
    u = 2.0 ** -24
    for (h, m, n, rp, co, vo), X, Xt, Yt in zip(mats, Xs, Xd, Yd):
        Y = Yt.cpu().numpy()
        L = np.diff(rp).astype(np.float64)
        ref = oracle.csr_spmm(rp, co, vo, X.astype(np.float64))
        for q in range(k):
            y1 = torch.empty(m, dtype=torch.float32, device=DEV)
            sp.spmv_mul(h, Xt[:, q].contiguous(), y1, accum=accv)
            torch.cuda.synchronize()
            assert np.array_equal(Y[:, q], y1.cpu().numpy()), (m, q)
            scale = oracle.csr_absmul(rp, co, vo, X[:, q].astype(np.float64))
            g = (L + 1) * u / (1 - (L + 1) * u)          # FP32 accumulation bound, the loosest mode
            assert (np.abs(Y[:, q] - ref[:, q]) <= g * scale + u * np.abs(ref[:, q])).all()
        sp.spmv_destroy(h)


def test_batch_replay_new_vectors_and_formats(sp):
    """Second call with the same shape replays the captured graph with new X / Y; handles
    converted to row-split or HB get their merge tiles on first use."""
    k = 4
    mats = build(sp, fmt="rowsplit")
    sp.spmv_convert(mats[1][0], "hb")
    hs = [t[0] for t in mats]
    for rep in range(3):
        Xs = [rhs(n, k, 500 + 10 * rep + i) for i, (_, m, n, *_r) in enumerate(mats)]
        Yd = [torch.full((m, k), float("nan"), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
        sp.spmv_mul_batch(hs, [torch.from_numpy(X).to(DEV) for X in Xs], Yd, k=k)
        torch.cuda.synchronize()
        for (h, m, n, rp, co, vo), X, Yt in zip(mats, Xs, Yd):
            Y = Yt.cpu().numpy()
            ref = oracle.csr_spmm(rp, co, vo, X)
            for q in range(k):
                scale = oracle.csr_absmul(rp, co, vo, X[:, q])
                assert (np.abs(Y[:, q] - ref[:, q]) <= TOL * scale).all(), (rep, m, q)
    # a subset of the handles is a different batch shape
    sub = [mats[0], mats[2]]
    Xs = [rhs(n, k, 900 + i) for i, (_, m, n, *_r) in enumerate(sub)]
    Yd = [torch.empty((m, k), dtype=torch.float64, device=DEV) for (_, m, *_r) in sub]
    sp.spmv_mul_batch([t[0] for t in sub], [torch.from_numpy(X).to(DEV) for X in Xs], Yd, k=k)
    torch.cuda.synchronize()
    for (h, m, n, rp, co, vo), X, Yt in zip(sub, Xs, Yd):
        ref = oracle.csr_spmm(rp, co, vo, X)
        scale = np.stack([oracle.csr_absmul(rp, co, vo, X[:, q]) for q in range(k)], axis=1)
        assert (np.abs(Yt.cpu().numpy() - ref) <= TOL * scale).all()
    for t in mats:
        sp.spmv_destroy(t[0])


def test_batch_unaligned_rows_use_scalar_gathers(sp):
    """X whose base is not 16-byte aligned (k = 4) takes the one-value-per-load path."""
    k = 4
    mats = build(sp)[:2]
    hs = [t[0] for t in mats]
    Xs = [rhs(n, k, 40 + i) for i, (_, m, n, *_r) in enumerate(mats)]
    bufs = [torch.empty(X.size + 1, dtype=torch.float64, device=DEV) for X in Xs]
    Xd = []
    for b, X in zip(bufs, Xs):
        v = b[1:].view(X.shape)
        v.copy_(torch.from_numpy(X))
        Xd.append(v)
    Yd = [torch.empty((m, k), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
    sp.spmv_mul_batch(hs, Xd, Yd, k=k)
    torch.cuda.synchronize()
    for (h, m, n, rp, co, vo), X, Yt in zip(mats, Xs, Yd):
        ref = oracle.csr_spmm(rp, co, vo, X)
        scale = np.stack([oracle.csr_absmul(rp, co, vo, X[:, q]) for q in range(k)], axis=1)
        assert (np.abs(Yt.cpu().numpy() - ref) <= TOL * scale).all()
        sp.spmv_destroy(h)


def test_batch_errors(sp):
    mats = build(sp)[:2]
    hs = [t[0] for t in mats]
    X = [torch.zeros((n, 2), dtype=torch.float64, device=DEV) for (_, m, n, *_r) in mats]
    Y = [torch.zeros((m, 2), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
    for bad_k in (0, 17):
        with pytest.raises(sp.SpmvError) as e:
            sp.spmv_mul_batch(hs, X, Y, k=bad_k)
        assert e.value.status == sp.SPMV_ERR_INVALID_ARG
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_mul_batch(hs, X, Y, k=2, accum=sp.SPMV_ACC_COMPENSATED)
    assert e.value.status == sp.SPMV_ERR_UNSUPPORTED
    r, c = synth.erdos_renyi(64, 3, seed=2)
    hp = sp.spmv_create_coo(64, 64, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV), None,
                            dtype=sp.SPMV_PATTERN)
    with pytest.raises(sp.SpmvError) as e:                       # not converted yet
        sp.spmv_mul_batch([hp], [X[0][:64]], [Y[0][:64]], k=2)
    assert e.value.status == sp.SPMV_ERR_NOT_CONVERTED
    sp.spmv_convert(hp, "merge")
    with pytest.raises(sp.SpmvError) as e:                       # mixed matrix dtypes
        sp.spmv_mul_batch([hs[0], hp], [X[0], X[0][:64]], [Y[0], Y[0][:64]], k=2)
    assert e.value.status == sp.SPMV_ERR_UNSUPPORTED
    sp.spmv_mul_batch([], [], [], k=2)                           # empty batch is a no-op
    for h in hs + [hp]:
        sp.spmv_destroy(h)


def test_tune_picks_a_measured_format(sp):
    scale = 14
    n = 1 << scale
    r, c = synth.rmat(scale, 16, seed=90)
    v = synth.values(r, c, 91)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV), torch.from_numpy(v).to(DEV))
    sp.spmv_convert(h, "rowsplit")
    res = sp.spmv_tune(h, "f64", hb=True)
    ms = res["ms"]
    assert all(t > 0 for t in ms.values()), ms
    assert set(ms) == {"rowsplit", "merge", "hb", "hb_chunked"}
    assert res["chosen"] == min(ms, key=ms.get)
    assert sp.spmv_info(h)["format"] == sp.FORMATS["hb" if res["chosen"].startswith("hb") else res["chosen"]]
    rp, co, vo = oracle.coo_to_csr(n, n, r, c, v)
    x = synth.vector(n, 92)
    y = torch.empty(n, dtype=torch.float64, device=DEV)
    sp.spmv_mul(h, torch.from_numpy(x).to(DEV), y)
    torch.cuda.synchronize()
    assert (np.abs(y.cpu().numpy() - oracle.csr_spmv(rp, co, vo, x)) <= TOL * oracle.csr_absmul(rp, co, vo, x)).all()
    # with Merge Blocking among the candidates: five timings, the choice the fastest, the product right
    res = sp.spmv_tune(h, "f64", hb=True, mergeb=True)
    ms = res["ms"]
    assert set(ms) == {"rowsplit", "merge", "hb", "hb_chunked", "mergeb"} and all(t > 0 for t in ms.values()), ms
    assert res["chosen"] == min(ms, key=ms.get)
    y.fill_(float("nan"))
    sp.spmv_mul(h, torch.from_numpy(x).to(DEV), y)
    torch.cuda.synchronize()
    assert (np.abs(y.cpu().numpy() - oracle.csr_spmv(rp, co, vo, x)) <= TOL * oracle.csr_absmul(rp, co, vo, x)).all()
    sp.spmv_destroy(h)


def test_batch_k1_runs_each_handles_active_format(sp):
    """k = 1: row-split and blocked handles run their own product (result = spmv_mul), the
    merge-path ones share the persistent launch."""
    mats = build(sp)
    sp.spmv_convert(mats[0][0], "rowsplit")
    sp.spmv_convert(mats[1][0], "hb")
    Xs = [rhs(n, 1, 60 + i) for i, (_, m, n, *_r) in enumerate(mats)]
    Xd = [torch.from_numpy(X).to(DEV) for X in Xs]
    Yd = [torch.full((m, 1), float("nan"), dtype=torch.float64, device=DEV) for (_, m, *_r) in mats]
    sp.spmv_mul_batch([t[0] for t in mats], Xd, Yd, k=1, accum=sp.SPMV_ACC_F64)
    torch.cuda.synchronize()
    for i, ((h, m, n, rp, co, vo), X, Xt, Yt) in enumerate(zip(mats, Xs, Xd, Yd)):
        y1 = torch.empty(m, dtype=torch.float64, device=DEV)
        sp.spmv_mul(h, Xt[:, 0].contiguous(), y1, accum=sp.SPMV_ACC_F64)
        torch.cuda.synchronize()
        got = Yt.cpu().numpy()[:, 0]
        if i != 1:   # the blocked product adds with atomics: equal within tolerance, not bitwise
            assert np.array_equal(got, y1.cpu().numpy()), i
        scale = oracle.csr_absmul(rp, co, vo, X[:, 0])
        assert (np.abs(got - oracle.csr_spmv(rp, co, vo, X[:, 0])) <= TOL * scale).all(), i
    for t in mats:
        sp.spmv_destroy(t[0])


@pytest.mark.parametrize("acc", ["F64", "SEGMENT"])
def test_batch_long_carry_runs_bitwise_equal_to_single(sp, acc):
    """Rows of up to 20,000 nonzeros span more than 16 warp tiles, so their carries are summed
    by the warp-wide fix-up; the batch must reproduce spmv_mul bit for bit there too."""
    n = 20000
    r, c = synth.zipf_rows(n, 1.2, n, 0.05, seed=95)
    perm = synth.shuffle_order(r.size, 6)
    r, c = r[perm], c[perm]
    v = synth.values(r, c, 96)
    f32 = acc == "SEGMENT"
    vd = torch.from_numpy(v.astype(np.float32) if f32 else v).to(DEV)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV), vd)
    sp.spmv_convert(h, "merge")
    accv = getattr(sp, "SPMV_ACC_" + acc)
    dt = np.float32 if f32 else np.float64
    for k in (1, 4):
        X = rhs(n, k, 97, dtype=dt)
        Xd = torch.from_numpy(X).to(DEV)
        Y = torch.full((n, k), float("nan"), dtype=Xd.dtype, device=DEV)
        sp.spmv_mul_batch([h], [Xd], [Y], k=k, accum=accv)
        torch.cuda.synchronize()
        for q in range(k):
            y1 = torch.empty(n, dtype=Xd.dtype, device=DEV)
            sp.spmv_mul(h, Xd[:, q].contiguous(), y1, accum=accv)
            torch.cuda.synchronize()
            assert np.array_equal(Y[:, q].cpu().numpy(), y1.cpu().numpy()), (k, q)
    sp.spmv_destroy(h)
