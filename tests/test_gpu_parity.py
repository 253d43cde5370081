"""Parity of the CUDA path (called through the C ABI) with the CPU oracle.

Integer, pattern, index and format results are compared bit for bit.  Floating-point
products must satisfy |y_i - y_ref,i| <= 1e-13 * (|A| |x|)_i against Algorithm 1.
Sizes span several CTA tiles with ragged tails; edge cases cover empty matrices, empty
rows, a single dense row, rows longer than a tile, rectangular shapes and bad input.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


DEV = "cuda:0"


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def make_handle(sp, m, n, rows, cols, vals, flags=0):
    return sp.spmv_create_coo(m, n, dev(rows), dev(cols), None if vals is None else dev(vals), flags=flags,
                              dtype=None if vals is not None else sp.SPMV_PATTERN)


def gpu_mul(sp, h, x, m, accum=0):
    xd = dev(x)
    y = torch.full((m,), float("nan"), dtype=xd.dtype, device=DEV)
    sp.spmv_mul(h, xd, y, accum=accum)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def check_float(y, rp, co, vo, x):
    ref = oracle.csr_spmv(rp, co, vo, x)
    scale = oracle.csr_absmul(rp, co, vo, x)
    err = np.abs(y - ref)
    assert np.isfinite(y).all()
    worst = np.max(err - TOL * scale) if y.size else 0
    assert (err <= TOL * scale).all(), f"max excess {worst}"


ALGOS = ["merge", "rowsplit", "hb"]


# ------------------------------------------------------------------ Hilbert key kernel

def test_hilbert_key_kernel_matches_oracle_and_figure(sp):
    from test_oracle_pins import hilbert_figure_tables
    tabs = hilbert_figure_tables()
    for K in range(1, 9):
        S = 1 << K
        r, c = np.meshgrid(np.arange(S, dtype=np.int32), np.arange(S, dtype=np.int32), indexing="ij")
        keys = torch.empty(S * S, dtype=torch.int64, device=DEV)
        sp.spmv_hilbert_keys(K, dev(r.ravel()), dev(c.ravel()), keys)
        got = keys.cpu().numpy().reshape(S, S)
        np.testing.assert_array_equal(got, oracle.hilbert_table(K))
        if K in tabs:
            np.testing.assert_array_equal(got, tabs[K])
    rng = np.random.default_rng(0)
    for K in (22, 31):
        r = rng.integers(0, 1 << K, 5000, dtype=np.int64).astype(np.int32)
        c = rng.integers(0, 1 << K, 5000, dtype=np.int64).astype(np.int32)
        keys = torch.empty(5000, dtype=torch.int64, device=DEV)
        sp.spmv_hilbert_keys(K, dev(r), dev(c), keys)
        got = keys.cpu().numpy().view(np.uint64)
        ref = np.array([oracle.hilbert_index(K, int(a), int(b)) for a, b in zip(r, c)], dtype=np.uint64)
        np.testing.assert_array_equal(got, ref)


# ------------------------------------------------------------------ COO -> CSR

CASES = [
    # (m, n, nnz, seed, dup_frac)
    (1, 1, 1, 0, 0.0),
    (1, 5000, 3000, 1, 0.0),        # one dense row (spans several merge tiles)
    (5000, 1, 3000, 2, 0.0),        # one dense column
    (37, 53, 400, 3, 0.0),
    (1000, 700, 9000, 4, 0.0),      # rectangular, several tiles
    (4097, 4097, 50000, 5, 0.0),    # ragged tails
    (3000, 3000, 20000, 6, 0.3),    # duplicates
    (70000, 70000, 30000, 7, 0.0),  # mostly empty rows
    (1, 200000, 150000, 8, 0.0),    # one row far longer than a shared-memory sort (per-row radix)
    (50, 100000, 200000, 9, 0.2),   # long rows with duplicates (ties kept in input order)
    (20000, 20000, 100000, 10, 0.3),  # short rows with duplicates
    (3, 5000, 6000, 11, 0.5),       # rows near the short/long boundary, many duplicates
]


@pytest.mark.parametrize("m,n,nnz,seed,dup", CASES)
def test_coo_to_csr_bit_exact(sp, m, n, nnz, seed, dup):
    rows, cols = synth.random_coo(m, n, nnz, seed, dup_frac=dup)
    vals = synth.values(rows, cols, seed) * (1 + np.arange(rows.size) % 3)   # duplicates differ
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "merge")
    rp, co, vo = sp.spmv_export_csr(h)
    orp, oco, ovo = oracle.coo_to_csr(m, n, rows, cols, vals)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(co, oco)
    np.testing.assert_array_equal(vo, ovo)
    assert sp.spmv_info(h)["nnz"] == oco.size


def test_coo_to_csr_rmat_and_host_input(sp):
    rows, cols = synth.rmat(14, 16, seed=3)
    m = n = 1 << 14
    vals = synth.values(rows, cols, 3)
    # host pointers (the library copies from host memory)
    h = sp.spmv_create_coo(m, n, rows, cols, vals)
    sp.spmv_convert(h, "rowsplit")
    rp, co, vo = sp.spmv_export_csr(h)
    orp, oco, ovo = oracle.coo_to_csr(m, n, rows, cols, vals)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(co, oco)
    np.testing.assert_array_equal(vo, ovo)


def test_pattern_and_empty(sp):
    rows, cols = synth.random_coo(300, 200, 1500, 11)
    h = make_handle(sp, 300, 200, rows, cols, None)
    sp.spmv_convert(h, "merge")
    rp, co, vo = sp.spmv_export_csr(h)
    orp, oco, _ = oracle.coo_to_csr(300, 200, rows, cols, None)
    np.testing.assert_array_equal(rp, orp)
    np.testing.assert_array_equal(co, oco)
    assert vo is None
    for fmt in ALGOS:
        for (m, n) in [(0, 0), (0, 5), (5, 0), (7, 9)]:
            e = np.zeros(0, np.int32)
            h = sp.spmv_create_coo(m, n, dev(e), dev(e), dev(np.zeros(0)))
            sp.spmv_convert(h, fmt)
            if m:
                y = gpu_mul(sp, h, np.ones(n), m)
                assert (y == 0).all()


def test_errors(sp):
    rows = np.array([0, 1, 5], np.int32)
    cols = np.array([0, 1, 1], np.int32)
    with pytest.raises(sp.SpmvError) as e:
        make_handle(sp, 4, 4, rows, cols, np.ones(3))
    assert e.value.status == sp.SPMV_ERR_INDEX_RANGE
    rows = np.array([0, 1, 1], np.int32)
    cols = np.array([0, 1, 1], np.int32)
    h = make_handle(sp, 4, 4, rows, cols, np.ones(3), flags=sp.SPMV_DUP_ERROR)
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_convert(h, "merge")
    assert e.value.status == sp.SPMV_ERR_DUPLICATE
    h = make_handle(sp, 4, 4, rows, cols, np.ones(3))
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_mul(h, dev(np.ones(4)), torch.empty(4, dtype=torch.float64, device=DEV))
    assert e.value.status == sp.SPMV_ERR_NOT_CONVERTED
    # host-side allocation failure injection: fails cleanly, library stays usable
    sp.spmv_test_fail_alloc(2)
    try:
        with pytest.raises(sp.SpmvError) as e:
            h2 = make_handle(sp, 4, 4, rows, cols, np.ones(3))
            sp.spmv_convert(h2, "merge")
        assert e.value.status == sp.SPMV_ERR_OOM
    finally:
        sp.spmv_test_fail_alloc(-1)
    sp.spmv_convert(h, "merge")
    y = gpu_mul(sp, h, np.ones(4), 4)
    np.testing.assert_array_equal(y, [1, 2, 0, 0])


# ------------------------------------------------------------------ merge partition

@pytest.mark.parametrize("scale", [8, 13])
def test_merge_partition_split_points(sp, scale):
    rows, cols = synth.rmat(scale, 16, seed=scale)
    m = n = 1 << scale
    h = make_handle(sp, m, n, rows, cols, synth.values(rows, cols, 0))
    sp.spmv_convert(h, "merge")
    rs, ns = sp.spmv_export_merge_partition(h)
    info = sp.spmv_info(h)
    orp, _, _ = oracle.coo_to_csr(m, n, rows, cols, None)
    T = info["merge_tile_items"]
    for t in range(info["merge_tiles"] + 1):
        d = min(t * T, m + int(orp[-1]))
        assert (rs[t], ns[t]) == oracle.merge_path_search(d, orp), t


# ------------------------------------------------------------------ SpMV parity

SPMV_CASES = [(1, 1, 1, 0), (1, 9000, 6000, 1), (9000, 1, 6000, 2), (37, 53, 400, 3), (1000, 700, 9000, 4),
              (4097, 4097, 50000, 5), (70000, 70000, 30000, 7), (20000, 20000, 400000, 8)]


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("m,n,nnz,seed", SPMV_CASES)
def test_spmv_integer_bit_exact(sp, algo, m, n, nnz, seed):
    rows, cols = synth.random_coo(m, n, nnz, seed)
    vals = synth.values(rows, cols, seed, integer=True)
    x = synth.vector(n, seed + 1, integer=True)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, algo)
    y = gpu_mul(sp, h, x, m)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    np.testing.assert_array_equal(y, oracle.csr_spmv(rp, co, vo, x))


@pytest.mark.parametrize("algo", ALGOS)
@pytest.mark.parametrize("m,n,nnz,seed", SPMV_CASES)
def test_spmv_float_tolerance(sp, algo, m, n, nnz, seed):
    rows, cols = synth.random_coo(m, n, nnz, seed)
    vals = synth.values(rows, cols, seed)
    x = synth.vector(n, seed + 1)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, algo)
    y = gpu_mul(sp, h, x, m)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    check_float(y, rp, co, vo, x)


@pytest.mark.parametrize("algo", ALGOS)
def test_spmv_rmat_scale16_both_variants(sp, algo):
    """R-MAT n = 2^16, edge factor 16, Graph500 a/b/c/d, deduplicated: U(-1,1) values
    within tolerance, and the integer-valued variant bit-exact."""
    rows, cols = synth.rmat(16, 16, seed=0)
    m = n = 1 << 16
    for integer in (False, True):
        vals = synth.values(rows, cols, 0, integer=integer)
        x = synth.vector(n, 1, integer=integer)
        h = make_handle(sp, m, n, rows, cols, vals)
        sp.spmv_convert(h, algo)
        y = gpu_mul(sp, h, x, m)
        rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
        if integer:
            np.testing.assert_array_equal(y, oracle.csr_spmv(rp, co, vo, x))
        else:
            check_float(y, rp, co, vo, x)
        # pattern variant (values implicitly 1) with integer x: exact
        hp = make_handle(sp, m, n, rows, cols, None)
        sp.spmv_convert(hp, algo)
        xi = synth.vector(n, 2, integer=True)
        np.testing.assert_array_equal(gpu_mul(sp, hp, xi, m), oracle.csr_spmv(rp, co, None, xi))


@pytest.mark.parametrize("algo", ALGOS)
def test_spmv_repeat_deterministic_and_invariants(sp, algo):
    rows, cols = synth.rmat(12, 16, seed=5)
    m = n = 1 << 12
    vals = synth.values(rows, cols, 5)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, algo)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    # A 1 = row sums
    y1 = gpu_mul(sp, h, np.ones(n), m)
    rs = oracle.csr_spmv(rp, co, vo, np.ones(n))
    assert (np.abs(y1 - rs) <= TOL * oracle.csr_absmul(rp, co, vo, np.ones(n))).all()
    # x^T (A y) = (A^T x)^T y with A^T from the oracle
    xv, yv = synth.vector(m, 7), synth.vector(n, 8)
    trp, tco, tvo = oracle.csr_transpose(m, n, rp, co, vo)
    lhs = float(np.dot(xv, gpu_mul(sp, h, yv, m)))
    rhs = float(np.dot(oracle.csr_spmv(trp, tco, tvo, xv), yv))
    bound = float(np.dot(np.abs(xv), oracle.csr_absmul(rp, co, vo, np.abs(yv))))
    assert abs(lhs - rhs) <= 1e-12 * bound
    if algo != "hb":   # CSR products use a fixed summation order: identical bits on repeat
        a = gpu_mul(sp, h, yv, m)
        b = gpu_mul(sp, h, yv, m)
        np.testing.assert_array_equal(a, b)


# ------------------------------------------------------------------ FP64 arithmetic paths

@pytest.mark.parametrize("algo", ["merge", "rowsplit"])
def test_fp64_native_and_double_float_paths(sp, algo):
    """SPMV_ACC_F64 (native FP64 pipe) and the default (double-float on FP32 pipes) both
    meet the tolerance; integer data is bit-exact on both."""
    rows, cols = synth.rmat(14, 16, seed=21)
    m = n = 1 << 14
    for integer in (False, True):
        vals = synth.values(rows, cols, 21, integer=integer)
        x = synth.vector(n, 22, integer=integer)
        rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
        h = make_handle(sp, m, n, rows, cols, vals)
        sp.spmv_convert(h, algo)
        for acc in (sp.SPMV_ACC_DEFAULT, sp.SPMV_ACC_F64):
            y = gpu_mul(sp, h, x, m, accum=acc)
            if integer:
                np.testing.assert_array_equal(y, oracle.csr_spmv(rp, co, vo, x))
            else:
                check_float(y, rp, co, vo, x)


@pytest.mark.parametrize("algo", ["merge", "rowsplit"])
def test_double_float_window_fallbacks(sp, algo):
    """Values outside [2^-50, 2^45] switch to native FP64: an x entry of 1e-20 (checked
    per product on the device) and a stored value of 1e300 (checked at conversion)."""
    rows, cols = synth.rmat(12, 16, seed=23)
    m = n = 1 << 12
    vals = synth.values(rows, cols, 23)
    x = synth.vector(n, 24)
    x_small = x.copy()
    x_small[cols[0]] = 1e-20
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, algo)
    check_float(gpu_mul(sp, h, x_small, m), rp, co, vo, x_small)
    check_float(gpu_mul(sp, h, x, m), rp, co, vo, x)        # flag cleared again on the next call
    big = vals.copy()
    big[0] = 1e300
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, big)
    h = make_handle(sp, m, n, rows, cols, big)
    sp.spmv_convert(h, algo)
    check_float(gpu_mul(sp, h, x, m), rp, co, vo, x)


# ------------------------------------------------------------------ CSR -> HB

@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("log2beta", [0, 3, 7])
def test_hb_structure_bit_exact(sp, inner, log2beta):
    for (m, n, scale) in [(1 << 12, 1 << 12, 12), (3000, 1700, None)]:
        if scale:
            rows, cols = synth.rmat(scale, 16, seed=9)
        else:
            rows, cols = synth.random_coo(m, n, 20000, 9)
        vals = synth.values(rows, cols, 9)
        h = make_handle(sp, m, n, rows, cols, vals)
        sp.spmv_convert(h, "hb", log2_beta=log2beta, inner_order=inner)
        got = sp.spmv_export_hb(h)
        rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
        lb = log2beta or oracle.log2_beta(n, 8, 200 * 1024)
        ref = oracle.csr_to_hb(m, n, rp, co, vo, lb, inner)
        assert got["nblk"] == ref["nblk"] and got["log2beta"] == ref["log2beta"]
        for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=k)
        # the product over the oracle's own blocked structure agrees too
        x = synth.vector(n, 3)
        y = gpu_mul(sp, h, x, m)
        yh = oracle.hb_spmv(m, ref, x)
        assert (np.abs(y - yh) <= TOL * oracle.csr_absmul(rp, co, vo, x)).all()


@pytest.mark.parametrize("inner", [0, 1])
def test_hb_product_integer_exact(sp, inner):
    """Integer values and x: the blocked product (runs of equal rows summed in the warp, then
    atomics in any order) is exact in both inner orders, on a hub-heavy R-MAT matrix."""
    rows, cols = synth.rmat(13, 32, seed=4)
    m = n = 1 << 13
    vals = synth.values(rows, cols, 4, integer=True)
    x = synth.vector(n, 5, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = make_handle(sp, m, n, rows, cols, vals)
    for lb in (0, 4, 9):
        sp.spmv_convert(h, "hb", log2_beta=lb, inner_order=inner)
        np.testing.assert_array_equal(gpu_mul(sp, h, x, m), ref)


def test_bounded_wait_gives_up_and_device_stays_usable(sp):
    """A kernel waiting on an mbarrier that nothing arrives at gives up after its poll limit,
    reports the timeout bit through the status word and returns; products run afterwards."""
    for polls in (1, 1000):
        assert sp.spmv_test_wait_timeout(polls) & 4
    rows, cols = synth.rmat(10, 8, seed=6)
    m = n = 1 << 10
    vals = synth.values(rows, cols, 6, integer=True)
    x = synth.vector(n, 6, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "merge")
    np.testing.assert_array_equal(gpu_mul(sp, h, x, m), oracle.csr_spmv(rp, co, vo, x))
    sp.spmv_wait(h)   # no product wait gave up


def test_formats_coexist_on_one_handle(sp):
    rows, cols = synth.rmat(11, 16, seed=2)
    m = n = 1 << 11
    vals = synth.values(rows, cols, 2, integer=True)
    x = synth.vector(n, 3, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = make_handle(sp, m, n, rows, cols, vals)
    for algo in ["rowsplit", "hb", "merge", "hb", "rowsplit"]:
        sp.spmv_convert(h, algo)
        np.testing.assert_array_equal(gpu_mul(sp, h, x, m), ref)


# ------------------------------------------------------------------ full size (bench launch configuration)

@pytest.mark.slow
def test_rmat_scale22_full_size(sp):
    """R-MAT scale 22 (the benchmark workload): CSR bit-exact against the oracle; every
    product algorithm within tolerance on all rows; the blocked arrays at beta = 2^14 bit-exact
    in both inner orders; the integer variant bit-exact for every product."""
    rows, cols = synth.rmat(22, 16, seed=0)
    m = n = 1 << 22
    vals = synth.values(rows, cols, 0)
    x = synth.vector(n, 1)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    scale = oracle.csr_absmul(rp, co, vo, x)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "merge")
    grp, gco, gvo = sp.spmv_export_csr(h)
    np.testing.assert_array_equal(grp, rp)
    np.testing.assert_array_equal(gco, co)
    np.testing.assert_array_equal(gvo, vo)
    for algo in ALGOS:
        sp.spmv_convert(h, algo)
        y = gpu_mul(sp, h, x, m)
        assert (np.abs(y - ref) <= TOL * scale).all(), algo
    # the blocked structure at the benchmark's block side 2^14 (K = 22), both inner orders,
    # bit for bit against the oracle's Hilbert sort (the curve's high levels included)
    for inner in (0, 1):
        sp.spmv_convert(h, "hb", log2_beta=14, inner_order=inner)
        got = sp.spmv_export_hb(h)
        want = oracle.csr_to_hb(m, n, rp, co, vo, 14, inner)
        assert got["nblk"] == want["nblk"] and got["log2beta"] == 14
        for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
            np.testing.assert_array_equal(got[k], want[k], err_msg=f"{k} inner={inner}")
        del got, want
    del h
    vi = synth.values(rows, cols, 0, integer=True)
    xi = synth.vector(n, 1, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vi)
    refi = oracle.csr_spmv(rp, co, vo, xi)
    h = make_handle(sp, m, n, rows, cols, vi)
    for algo in ALGOS:
        sp.spmv_convert(h, algo)
        np.testing.assert_array_equal(gpu_mul(sp, h, xi, m), refi, err_msg=algo)
    sp.spmv_convert(h, "hb", inner_order=1)
    np.testing.assert_array_equal(gpu_mul(sp, h, xi, m), refi, err_msg="hb row-major inner order")


@pytest.mark.parametrize("log2beta", [9, 14])
@pytest.mark.parametrize("inner", [0, 1])
def test_hb_structure_rmat_scale17(sp, log2beta, inner):
    """Mid-size R-MAT (scale 17, K = 17): the blocked arrays bit for bit against the oracle
    at a small and at the benchmark's block side, and the integer product exact."""
    rows, cols = synth.rmat(17, 16, seed=17)
    m = n = 1 << 17
    vals = synth.values(rows, cols, 17, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = make_handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "hb", log2_beta=log2beta, inner_order=inner)
    got = sp.spmv_export_hb(h)
    want = oracle.csr_to_hb(m, n, rp, co, vo, log2beta, inner)
    assert got["nblk"] == want["nblk"]
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    x = synth.vector(n, 18, integer=True)
    np.testing.assert_array_equal(gpu_mul(sp, h, x, m), oracle.csr_spmv(rp, co, vo, x))
