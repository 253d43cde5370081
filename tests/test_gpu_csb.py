"""Compressed sparse blocks with row-major block order (CSB with the Z-Morton inner order,
Section 3.1; CSBH with the block's own Hilbert curve, Section 4.1), through the C ABI: the
blocked arrays bit for bit against the oracle, products exact on integer data with both HB
products, and the Z-Morton order with Hilbert-ordered blocks too."""
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


def mul(sp, h, x, m):
    y = torch.full((m,), float("nan"), dtype=torch.float64, device=DEV)
    sp.spmv_mul(h, torch.from_numpy(x).to(DEV), y)
    torch.cuda.synchronize()
    return y.cpu().numpy()


CASES = [(14, 16, 0), (13, 32, 9), (12, 8, 4)]   # (scale, edge factor, log2 beta; 0 = Eq. 2)


@pytest.mark.parametrize("scale,ef,lb", CASES)
@pytest.mark.parametrize("border,inner", [(1, 2), (1, 0), (1, 1), (0, 2)])
def test_blocked_orders_bit_exact(sp, scale, ef, lb, border, inner):
    rows, cols = synth.rmat(scale, ef, seed=scale + ef)
    m = n = 1 << scale
    vals = synth.values(rows, cols, 3, integer=True)
    x = synth.vector(n, 4, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = sp.spmv_create_coo(m, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "hb", log2_beta=lb, inner_order=inner, block_order=border, hb_product=sp.SPMV_HB_CHUNKED)
    got = sp.spmv_export_hb(h)
    beta = lb or oracle.log2_beta(n, 8, 200 * 1024)
    if border == 1:
        want = oracle.csr_to_hb(m, n, rp, co, vo, beta, inner, block_order=1)
    else:   # Hilbert-ordered blocks, Z-Morton inside: sort the oracle's HB blocks' entries by Z-Morton
        want = oracle.csr_to_hb(m, n, rp, co, vo, beta, 1)
        zt = oracle.zmorton_table(want["log2beta"])
        idx, val = want["idx"].copy(), want["val"].copy()
        for t in range(want["nblk"]):
            a, b = want["blk_ptr"][t], want["blk_ptr"][t + 1]
            key = [zt[int(v) >> 16, int(v) & 0xFFFF] for v in idx[a:b]]
            o = np.argsort(key, kind="stable")
            idx[a:b], val[a:b] = idx[a:b][o], val[a:b][o]
        want["idx"], want["val"] = idx, val
    assert got["nblk"] == want["nblk"]
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
        np.testing.assert_array_equal(got[k], want[k], err_msg=k)
    assert sp.spmv_info(h)["hb_orders"] == 16 * border + inner
    np.testing.assert_array_equal(mul(sp, h, x, m), ref)                 # chunked product
    sp.spmv_convert(h, "hb", log2_beta=lb, inner_order=inner, block_order=border)
    np.testing.assert_array_equal(mul(sp, h, x, m), ref)                 # staged product
    sp.spmv_destroy(h)


def test_csb_shorthand_and_float(sp):
    """spmv_convert(h, "csb") is the row-major block order with the Z-Morton inner order; FP64
    products stay within 1e-13 (|A||x|)."""
    rows, cols = synth.rmat(14, 16, seed=8)
    n = 1 << 14
    vals = synth.values(rows, cols, 8)
    x = synth.vector(n, 9)
    rp, co, vo = oracle.coo_to_csr(n, n, rows, cols, vals)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "csb", hb_product=sp.SPMV_HB_CHUNKED)
    assert sp.spmv_info(h)["hb_orders"] == 16 * 1 + 2
    y = mul(sp, h, x, n)
    assert (np.abs(y - oracle.csr_spmv(rp, co, vo, x)) <= 1e-13 * oracle.csr_absmul(rp, co, vo, x)).all()
    sp.spmv_destroy(h)
