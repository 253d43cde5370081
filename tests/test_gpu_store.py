"""Converted formats kept on disk (spmv_save / spmv_load), through the C ABI: a loaded handle
multiplies exactly as the saved one (integer data bit for bit against the oracle, in every
format and both HB products), its CRS and blocked arrays equal the saved ones, and damaged or
foreign files are rejected with an error instead of being used."""
import os

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


@pytest.mark.parametrize("fmt,hbp", [("merge", 0), ("rowsplit", 0), ("hb", 0), ("hb", 1)])
def test_save_load_round_trip(sp, tmp_path, fmt, hbp):
    rows, cols = synth.rmat(13, 16, seed=51)
    m = n = 1 << 13
    vals = synth.values(rows, cols, 51, integer=True)
    x = synth.vector(n, 52, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    ref = oracle.csr_spmv(rp, co, vo, x)
    h = sp.spmv_create_coo(m, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "hb", log2_beta=9)
    sp.spmv_convert(h, fmt, log2_beta=9, hb_product=hbp)
    path = str(tmp_path / "a.spmv")
    sp.spmv_save(h, path)
    g = sp.spmv_load(path)
    assert sp.spmv_info(g)["format"] == sp.spmv_info(h)["format"]
    np.testing.assert_array_equal(mul(sp, g, x, m), ref)
    for a, b in zip(sp.spmv_export_csr(g), sp.spmv_export_csr(h)):
        np.testing.assert_array_equal(a, b)
    ga, ha = sp.spmv_export_hb(g), sp.spmv_export_hb(h)
    for k in ("idx", "val", "blk_ptr", "blk_row", "blk_col"):
        np.testing.assert_array_equal(ga[k], ha[k], err_msg=k)
    for other in ("merge", "rowsplit", "hb"):     # every format from the loaded arrays
        sp.spmv_convert(g, other, log2_beta=9)
        np.testing.assert_array_equal(mul(sp, g, x, m), ref, err_msg=other)
    sp.spmv_destroy(g)
    sp.spmv_destroy(h)


def test_damaged_and_foreign_files_are_rejected(sp, tmp_path):
    rows, cols = synth.rmat(10, 8, seed=53)
    n = 1 << 10
    vals = synth.values(rows, cols, 53)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "hb")
    path = str(tmp_path / "b.spmv")
    sp.spmv_save(h, path)
    blob = open(path, "rb").read()
    bad = bytearray(blob)
    bad[len(bad) // 2] ^= 0x40                      # one flipped bit inside the arrays
    (tmp_path / "flip.spmv").write_bytes(bytes(bad))
    (tmp_path / "short.spmv").write_bytes(blob[: len(blob) // 3])
    (tmp_path / "foreign.spmv").write_bytes(b"NOTAFILE" + blob[8:])
    for name, status in (("flip.spmv", sp.SPMV_ERR_IO), ("short.spmv", sp.SPMV_ERR_IO),
                         ("foreign.spmv", sp.SPMV_ERR_INVALID_ARG), ("missing.spmv", sp.SPMV_ERR_IO)):
        with pytest.raises(sp.SpmvError) as e:
            sp.spmv_load(str(tmp_path / name))
        assert e.value.status == status, name
    e2 = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                            torch.from_numpy(vals).to(DEV))
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_save(e2, str(tmp_path / "c.spmv"))   # nothing converted yet
    assert e.value.status == sp.SPMV_ERR_NOT_CONVERTED
    sp.spmv_destroy(h)
    sp.spmv_destroy(e2)
