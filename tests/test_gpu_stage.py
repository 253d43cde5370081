"""The staged blocked product (HB format, x slices of the block columns held in shared
memory), called through the C ABI, against the oracle.

Integer data is compared bit for bit (every partial sum is an integer below 2^53, so the
order of the row reductions does not matter); FP64 data within 1e-13 (|A| |x|)_i.  The cases
exercise what the layout has to get right: row gaps wider than the delta field (filler
entries), slices staged and slices gathered in one product, a last slice narrower than the
block side with an odd length, an x that is not 16-byte aligned, x outside the double-float
window, and agreement with the Hilbert-ordered chunk product on the same handle.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-13
DEV = "cuda:0"


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def mul(sp, h, x, m, accum=0, offset=0):
    """y = A x; `offset` > 0 places x at that many elements into a larger buffer (unaligned)."""
    buf = torch.zeros(x.size + offset, dtype=torch.float64, device=DEV)
    buf[offset:] = dev(x)
    xd = buf[offset:]
    y = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
    sp.spmv_mul(h, xd, y, accum=accum)
    torch.cuda.synchronize()
    return y.cpu().numpy()


def within(y, rp, co, vo, x):
    ref = oracle.csr_spmv(rp, co, vo, x)
    scale = oracle.csr_absmul(rp, co, vo, x)
    assert np.isfinite(y).all()
    assert (np.abs(y - ref) <= TOL * scale).all(), float(np.max(np.abs(y - ref) - TOL * scale))


@pytest.mark.parametrize("log2beta", [14, 16])
def test_row_gaps_wider_than_the_delta_field(sp, log2beta):
    """With 2^lb-wide slices a row delta has 32 - lb bits: gaps of 2^20 rows in one slice
    (beyond the 2^18 - 2 or 2^16 - 2 a word holds) go through filler entries."""
    m, n = 1 << 21, 1 << 17
    rng = np.random.default_rng(3)
    rows = [0, 1, 300000, 300001, 1200000, 2097151, 5, 70000, 1 << 20]
    cols = [7, 7, 7, 9, 7, 7, (1 << 16) + 3, (1 << 16) + 3, (1 << 16) + 3]
    r2 = rng.integers(0, m, 20000)
    c2 = rng.integers(0, n, 20000)
    rows = np.concatenate([rows, r2]).astype(np.int32)
    cols = np.concatenate([cols, c2]).astype(np.int32)
    vals = synth.values(rows, cols, 5, integer=True)
    x = synth.vector(n, 6, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
    sp.spmv_convert(h, "hb", log2_beta=log2beta)
    np.testing.assert_array_equal(mul(sp, h, x, m), oracle.csr_spmv(rp, co, vo, x))
    np.testing.assert_array_equal(mul(sp, h, x, m, accum=sp.SPMV_ACC_F64), oracle.csr_spmv(rp, co, vo, x))


def test_staged_and_gathered_slices_ragged_last_slice(sp):
    """n = 100003: dense slices are staged, sparse ones gathered, and the last slice holds
    an odd number of columns (the copy's scalar tail)."""
    m = n = 100003
    rng = np.random.default_rng(11)
    # power-law columns: a few slices carry most entries
    cols = np.minimum((rng.pareto(1.2, 2_000_000) * 2000).astype(np.int64), n - 1).astype(np.int32)
    rows = rng.integers(0, m, cols.size).astype(np.int32)
    cols[:5000] = n - 1 - rng.integers(0, 3, 5000)     # entries in the last, narrow slice
    for integer in (True, False):
        vals = synth.values(rows, cols, 12, integer=integer)
        x = synth.vector(n, 13, integer=integer)
        rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
        h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
        sp.spmv_convert(h, "hb")
        for acc in (sp.SPMV_ACC_DEFAULT, sp.SPMV_ACC_F64):
            for off in (0, 1):
                y = mul(sp, h, x, m, accum=acc, offset=off)
                if integer:
                    np.testing.assert_array_equal(y, oracle.csr_spmv(rp, co, vo, x))
                else:
                    within(y, rp, co, vo, x)


def test_x_outside_double_float_window(sp):
    """An x entry of 1e-20 makes the product switch to native FP64 on the device."""
    rows, cols = synth.rmat(14, 16, seed=23)
    m = n = 1 << 14
    vals = synth.values(rows, cols, 23)
    x = synth.vector(n, 24)
    x[cols[0]] = 1e-20
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
    sp.spmv_convert(h, "hb")
    within(mul(sp, h, x, m), rp, co, vo, x)
    x2 = synth.vector(n, 25)
    within(mul(sp, h, x2, m), rp, co, vo, x2)        # back on the double-float path


def test_double_float_window_edge_subnormal_parts(sp):
    """Values and x near the bottom of the double-float window (2^-50, exactly representable in
    FP32): products near 2^-100 whose rounding errors, the compensation parts of the run sums,
    are often subnormal floats.  Those take the exact widening (a short one covers normal numbers
    and zeros only); flushing them would leave errors near 2^-126, far above the tolerance of
    about 2^-140 at this scale."""
    rows, cols = synth.rmat(14, 16, seed=31)
    m = n = 1 << 14
    rng = np.random.default_rng(32)
    def near(k):
        v = np.ldexp(1.0 + rng.random(k), -50).astype(np.float32).astype(np.float64)
        return np.where(rng.random(k) < 0.5, -v, v)
    vals = near(rows.size)
    x = near(n)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
    sp.spmv_convert(h, "hb")
    y = mul(sp, h, x, m)
    within(y, rp, co, vo, x)
    # the compensation parts really are subnormal here: products of two such floats have
    # rounding errors below 2^-126 for a sizeable share of the pairs
    a = np.float32(vals[:1000])
    b = np.float32(x[cols[:1000]])
    err = a.astype(np.float64) * b.astype(np.float64) - (a * b).astype(np.float64)
    assert np.mean((err != 0) & (np.abs(err) < 2.0 ** -126)) > 0.1


@pytest.mark.parametrize("inner", [0, 1])
def test_staged_equals_chunked_product(sp, inner):
    """Both HB products on one handle agree bit for bit on integer data, at several block
    sides; the blocked arrays stay those of the Hilbert conversion."""
    rows, cols = synth.rmat(15, 16, seed=41)
    m = n = 1 << 15
    vals = synth.values(rows, cols, 41, integer=True)
    x = synth.vector(n, 42, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
    for lb in (0, 6, 12, 15):
        sp.spmv_convert(h, "hb", log2_beta=lb, inner_order=inner)
        a = mul(sp, h, x, m)
        sp.spmv_convert(h, "hb", log2_beta=lb, inner_order=inner, hb_product=sp.SPMV_HB_CHUNKED)
        b = mul(sp, h, x, m)
        np.testing.assert_array_equal(a, ref)
        np.testing.assert_array_equal(b, ref)
    got = sp.spmv_export_hb(h)
    want = oracle.csr_to_hb(m, n, rp, co, vo, 15, inner)
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)


def test_rmat_scale18_fp64(sp):
    """R-MAT scale 18 (several hundred tiles per hot slice): FP64 within tolerance, the
    pattern variant exact on integer x."""
    rows, cols = synth.rmat(18, 16, seed=7)
    m = n = 1 << 18
    vals = synth.values(rows, cols, 7)
    x = synth.vector(n, 8)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = sp.spmv_create_coo(m, n, dev(rows), dev(cols), dev(vals))
    sp.spmv_convert(h, "hb")
    within(mul(sp, h, x, m), rp, co, vo, x)
    hp = sp.spmv_create_coo(m, n, dev(rows), dev(cols), None, dtype=sp.SPMV_PATTERN)
    sp.spmv_convert(hp, "hb")
    xi = synth.vector(n, 9, integer=True)
    np.testing.assert_array_equal(mul(sp, hp, xi, m), oracle.csr_spmv(rp, co, None, xi))
