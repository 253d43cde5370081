"""Merge Blocking (MergeB and MergeBH, Section 4.3) through the C ABI, against the oracle: the
blocked arrays, the CRS pointer over blocks and every lane's merge-path split point bit for
bit; products exact on integer and pattern data and within 1e-13 (|A||x|) in FP64; FP32
vectors within the FP32 bound; edge cases (empty, one entry, one dense row or column,
non-square and ragged shapes, block rows without blocks); save/load; the batch with k = 1;
the benchmark's R-MAT scale 22 at beta = 2^14."""
import os
import tempfile

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"
TOL = 1e-13
U = 2.0 ** -24


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


def handle(sp, m, n, rows, cols, vals, dtype=None):
    v = torch.from_numpy(vals).to(DEV) if vals is not None else None
    return sp.spmv_create_coo(m, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV), v,
                              dtype=dtype)


def mul(sp, h, x, m, dt=torch.float64, acc=0):
    y = torch.full((m,), float("nan"), dtype=dt, device=DEV)
    sp.spmv_mul(h, torch.from_numpy(x).to(DEV), y, accum=acc)
    torch.cuda.synchronize()
    return y.cpu().numpy().astype(np.float64)


def lane_splits(mb, nnz):
    """Oracle split point of every lane's first item: the merge-path search of Section 3.3 over
    the block-row ends counted in entries, and the block holding that entry."""
    bp, rptr = mb["blk_ptr"], mb["blk_row_ptr"]
    ends = bp[rptr].astype(np.int32)                      # entries before block row i (i = 0..nbr)
    total = mb["nbr"] + nnz
    tiles = -(-total // 256)
    ent, blk = [], []
    for g in range(tiles * 32):
        _, e = oracle.merge_path_search(min(8 * g, total), ends)
        ent.append(e)
        blk.append(int(np.searchsorted(bp, e, side="right")) - 1 if e < nnz else mb["nblk"])
    return np.array(ent, np.int32), np.array(blk, np.int32)


CASES = [(12, 8, 4, 0), (12, 8, 4, 1), (13, 16, 9, 1), (13, 16, 9, 0), (11, 32, 0, 1)]


@pytest.mark.parametrize("scale,ef,lb,inner", CASES)
def test_mergeb_structure_and_products(sp, scale, ef, lb, inner):
    rows, cols = synth.rmat(scale, ef, seed=scale * 3 + inner)
    m = n = 1 << scale
    vals = synth.values(rows, cols, 11, integer=True)
    x = synth.vector(n, 12, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    h = handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "mergeb", log2_beta=lb, inner_order=inner)
    beta = lb or oracle.log2_beta(n, 8, 200 * 1024)
    want = oracle.csr_to_mergeb(m, n, rp, co, vo, beta, inner)
    got = sp.spmv_export_mergeb(h)
    info = sp.spmv_info(h)
    assert info["format"] == sp.SPMV_FMT_MERGEB and info["hb_orders"] == 16 + inner
    assert got["nblk"] == want["nblk"] and got["nbr"] == want["nbr"] and got["log2beta"] == want["log2beta"]
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col", "blk_row_ptr"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    ent, blk = lane_splits(want, int(rp[-1]))
    np.testing.assert_array_equal(got["lane_entry"], ent)
    np.testing.assert_array_equal(got["lane_block"], blk)
    ref = oracle.mergeb_spmv(m, want, x, parts=37)
    np.testing.assert_array_equal(ref, oracle.csr_spmv(rp, co, vo, x))
    np.testing.assert_array_equal(mul(sp, h, x, m), ref)
    # FP64 values: within the tolerance
    vf = synth.values(rows, cols, 13)
    xf = synth.vector(n, 14)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vf)
    hf = handle(sp, m, n, rows, cols, vf)
    sp.spmv_convert(hf, "mergeb", log2_beta=lb, inner_order=inner)
    y = mul(sp, hf, xf, m)
    assert (np.abs(y - oracle.csr_spmv(rp, co, vo, xf)) <= TOL * oracle.csr_absmul(rp, co, vo, xf)).all()
    sp.spmv_destroy(h)
    sp.spmv_destroy(hf)


def _coo(rows, cols):
    return np.asarray(rows, np.int32), np.asarray(cols, np.int32)


EDGE = {
    "one_entry": (5, 7, _coo([3], [6])),
    "dense_row": (1, 9000, _coo(np.zeros(9000), np.arange(9000))),
    "dense_col": (9000, 1, _coo(np.arange(9000), np.zeros(9000))),
    "wide_ragged": (37, 5000, synth.random_coo(37, 5000, 4000, 21)),
    "tall_ragged": (5000, 37, synth.random_coo(5000, 37, 4000, 22)),
    "empty_block_rows": (4096, 4096, _coo(np.r_[np.zeros(50), np.full(50, 4095)], np.r_[np.arange(50), np.arange(50)])),
}


@pytest.mark.parametrize("name", sorted(EDGE))
@pytest.mark.parametrize("inner", [0, 1])
def test_mergeb_edge_cases(sp, name, inner):
    m, n, (rows, cols) = EDGE[name]
    vals = synth.values(rows, cols, 31, integer=True)
    x = synth.vector(n, 32, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    for lb in (2, 5, 0):
        h = handle(sp, m, n, rows, cols, vals)
        sp.spmv_convert(h, "mergeb", log2_beta=lb, inner_order=inner)
        got = sp.spmv_export_mergeb(h)
        want = oracle.csr_to_mergeb(m, n, rp, co, vo, got["log2beta"], inner)
        for k in ("idx", "blk_ptr", "blk_row", "blk_col", "blk_row_ptr"):
            np.testing.assert_array_equal(got[k], want[k], err_msg=f"{k} lb={lb}")
        np.testing.assert_array_equal(mul(sp, h, x, m), ref, err_msg=f"lb={lb}")
        sp.spmv_destroy(h)
    hp = handle(sp, m, n, rows, cols, None, dtype=sp.SPMV_PATTERN)
    sp.spmv_convert(hp, "mergebh" if inner == 0 else "mergeb", log2_beta=3)
    np.testing.assert_array_equal(mul(sp, hp, x, m), oracle.csr_spmv(rp, co, None, x))
    sp.spmv_destroy(hp)


def test_mergeb_empty_and_errors(sp):
    r = np.zeros(0, np.int32)
    h = handle(sp, 10, 12, r, r, np.zeros(0))
    sp.spmv_convert(h, "mergeb")
    np.testing.assert_array_equal(mul(sp, h, np.ones(12), 10), np.zeros(10))
    assert sp.spmv_info(h)["nblk"] == 0
    sp.spmv_destroy(h)
    rows, cols = synth.rmat(10, 8, seed=3)
    h = handle(sp, 1 << 10, 1 << 10, rows, cols, synth.values(rows, cols, 3))
    sp.spmv_convert(h, "mergeb")
    y = torch.zeros(1 << 10, dtype=torch.float32, device=DEV)
    with pytest.raises(sp.SpmvError) as e:   # FP64 values with FP32 vectors
        sp.spmv_mul(h, torch.zeros(1 << 10, dtype=torch.float32, device=DEV), y)
    assert e.value.status == sp.SPMV_ERR_UNSUPPORTED
    sp.spmv_destroy(h)


@pytest.mark.parametrize("kind", ["f32", "bf16"])
def test_mergeb_fp32_vectors(sp, kind):
    """FP32 vectors: plain FP32 runs and compensated runs, both joined by FP32 reductions in y,
    so both keep the FP32 bound gamma(L + 1) (|A||x|) + u |ref| for any order of additions."""
    rows, cols = synth.rmat(13, 16, seed=41)
    m = n = 1 << 13
    vals64 = synth.values(rows, cols, 42)
    if kind == "f32":
        v = vals64.astype(np.float32)
        vd, v64 = torch.from_numpy(v).to(DEV), v.astype(np.float64)
    else:
        bits = synth.round_bf16_bits(vals64)
        vd, v64 = torch.from_numpy(bits.view(np.int16)).to(DEV).view(torch.bfloat16), synth.bf16_bits_to_float64(bits)
    x32 = synth.vector(n, 43).astype(np.float32)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, v64)
    ref = oracle.csr_spmv(rp, co, vo, x32.astype(np.float64))
    scale = oracle.csr_absmul(rp, co, vo, x32.astype(np.float64))
    L = np.diff(rp).astype(np.float64)
    g = (L + 1) * U / (1 - (L + 1) * U)
    h = sp.spmv_create_coo(m, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV), vd)
    for fmt in ("mergeb", "mergebh"):
        sp.spmv_convert(h, fmt)
        for acc in (sp.SPMV_ACC_F32, sp.SPMV_ACC_COMPENSATED):
            y = mul(sp, h, x32, m, dt=torch.float32, acc=acc)
            assert (np.abs(y - ref) <= g * scale + U * np.abs(ref)).all(), (fmt, acc)
    sp.spmv_destroy(h)


def test_mergeb_save_load_batch_and_reconvert(sp):
    rows, cols = synth.rmat(12, 16, seed=51)
    m = n = 1 << 12
    vals = synth.values(rows, cols, 52, integer=True)
    x = synth.vector(n, 53, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "mergeb", log2_beta=6)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "a.spmv")
        sp.spmv_save(h, path)
        h2 = sp.spmv_load(path)
    assert sp.spmv_info(h2)["format"] == sp.SPMV_FMT_MERGEB
    a, b = sp.spmv_export_mergeb(h), sp.spmv_export_mergeb(h2)
    for k in ("idx", "blk_ptr", "blk_row_ptr", "lane_entry", "lane_block"):
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    np.testing.assert_array_equal(mul(sp, h2, x, m), ref)
    # batch with k = 1 runs the handle's own product
    X = [torch.from_numpy(x).to(DEV), torch.from_numpy(x).to(DEV)]
    Y = [torch.zeros(m, dtype=torch.float64, device=DEV) for _ in range(2)]
    sp.spmv_mul_batch([h, h2], X, Y, k=1)
    torch.cuda.synchronize()
    for y in Y:
        np.testing.assert_array_equal(y.cpu().numpy(), ref)
    # an HB conversion in Hilbert block order replaces the blocked arrays (and drops the tables)
    sp.spmv_convert(h, "hb", log2_beta=6)
    assert sp.spmv_info(h)["mergeb_tiles"] == 0
    np.testing.assert_array_equal(mul(sp, h, x, m), ref)
    sp.spmv_convert(h, "mergeb", log2_beta=6)
    np.testing.assert_array_equal(mul(sp, h, x, m), ref)
    sp.spmv_destroy(h)
    sp.spmv_destroy(h2)


def test_mergeb_rmat_scale22_full_size(sp):
    """The benchmark workload (R-MAT scale 22, 65.2 M nonzeros) at beta = 2^14: the MergeB
    arrays and block-row pointer bit for bit, every lane split point on a sample of 4096 lanes,
    FP64 products within tolerance on every row for MergeB and MergeBH, integer products exact."""
    rows, cols = synth.rmat(22, 16, seed=0)
    m = n = 1 << 22
    vals = synth.values(rows, cols, 0)
    x = synth.vector(n, 1)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    scale = oracle.csr_absmul(rp, co, vo, x)
    h = handle(sp, m, n, rows, cols, vals)
    sp.spmv_convert(h, "mergeb", log2_beta=14)
    got = sp.spmv_export_mergeb(h)
    want = oracle.csr_to_mergeb(m, n, rp, co, vo, 14, 1)
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col", "blk_row_ptr"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    nnz = int(rp[-1])
    ends = want["blk_ptr"][want["blk_row_ptr"]].astype(np.int32)
    total = want["nbr"] + nnz
    rng = np.random.default_rng(7)
    lanes = got["lane_entry"].size
    for g in np.r_[0, lanes - 1, rng.integers(0, lanes, 4094)]:
        _, e = oracle.merge_path_search(min(8 * int(g), total), ends)
        assert got["lane_entry"][g] == e
        assert got["lane_block"][g] == (np.searchsorted(want["blk_ptr"], e, side="right") - 1 if e < nnz else want["nblk"])
    del got, want
    y = mul(sp, h, x, m)
    assert (np.abs(y - ref) <= TOL * scale).all()
    sp.spmv_convert(h, "mergebh", log2_beta=14)
    y = mul(sp, h, x, m)
    assert (np.abs(y - ref) <= TOL * scale).all()
    sp.spmv_destroy(h)
    vi = synth.values(rows, cols, 0, integer=True)
    xi = synth.vector(n, 1, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vi)
    h = handle(sp, m, n, rows, cols, vi)
    sp.spmv_convert(h, "mergeb", log2_beta=14)
    np.testing.assert_array_equal(mul(sp, h, xi, m), oracle.csr_spmv(rp, co, vo, xi))
    sp.spmv_destroy(h)
