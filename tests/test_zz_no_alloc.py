"""The allocation-free product spmv_mul_csr_merge_noalloc, called through the C ABI.

Some callers cannot allocate device memory while they run (for example inside an allocator
that owns all device memory, under a memory budget enforced outside the library, or in a
serving loop that must not pay the device synchronisation of cudaMalloc/cudaFree).  For them the library offers a
merge-path product whose scratch lives in a fixed array inside the library.  This test
checks it against the regular entry point (spmv_create_coo + spmv_convert + spmv_mul) and
against the oracle on two calls in a row, within the tolerance the other parity tests use,
bit for bit on integer data, and that an oversized input is rejected.  The file name sorts last so that a run stopping at the
first failure has already run every other test.
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


def test_noalloc_matches_regular_entry_point_twice(sp):
    dev = "cuda:0"
    scale = 16
    m = n = 1 << scale
    rows, cols = synth.rmat(scale, 16, seed=31)
    vals = synth.values(rows, cols, 31)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    nnz = int(rp[-1])
    rp_d, co_d, vo_d = (torch.from_numpy(a).to(dev) for a in (rp, co, vo))
    h = sp.spmv_create_coo(m, n, *(torch.from_numpy(a).to(dev) for a in (rows, cols, vals)))
    sp.spmv_convert(h, "merge")
    lib = sp._lib
    stream = torch.cuda.current_stream().cuda_stream
    for call, seed in enumerate((41, 42)):          # two calls in a row, different x
        x = synth.vector(n, seed)
        x_d = torch.from_numpy(x).to(dev)
        y_ref = torch.empty(m, dtype=torch.float64, device=dev)
        sp.spmv_mul(h, x_d, y_ref)
        y_new = torch.full((m,), float("nan"), dtype=torch.float64, device=dev)
        st = lib.spmv_mul_csr_merge_noalloc(m, n, nnz, rp_d.data_ptr(), co_d.data_ptr(), vo_d.data_ptr(),
                                            x_d.data_ptr(), y_new.data_ptr(), stream)
        assert st == sp.SPMV_OK, sp.spmv_last_error()
        torch.cuda.synchronize()
        a, b = y_new.cpu().numpy(), y_ref.cpu().numpy()
        scale_abs = oracle.csr_absmul(rp, co, vo, x)
        assert np.isfinite(a).all(), f"call {call}"
        assert (np.abs(a - b) <= TOL * scale_abs).all(), f"call {call}"
        assert (np.abs(a - oracle.csr_spmv(rp, co, vo, x)) <= TOL * scale_abs).all(), f"call {call}"
    sp.spmv_destroy(h)


def test_noalloc_integer_bit_exact_against_oracle(sp):
    """Integer values and x: every partial sum is an integer below 2^53, so two calls in a
    row (the shared scratch holding the first call's partition and carries) equal the
    oracle's Algorithm 1 bit for bit."""
    dev = "cuda:0"
    m, n = 30011, 29989                              # ragged: no multiple of the tile size
    rows, cols = synth.rmat(15, 16, seed=33)
    keep = (rows < m) & (cols < n)
    rows, cols = rows[keep], cols[keep]
    vals = synth.values(rows, cols, 33, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals)
    nnz = int(rp[-1])
    rp_d, co_d, vo_d = (torch.from_numpy(a).to(dev) for a in (rp, co, vo))
    stream = torch.cuda.current_stream().cuda_stream
    for seed in (51, 52):
        x = synth.vector(n, seed, integer=True)
        x_d = torch.from_numpy(x).to(dev)
        y = torch.full((m,), float("nan"), dtype=torch.float64, device=dev)
        st = sp._lib.spmv_mul_csr_merge_noalloc(m, n, nnz, rp_d.data_ptr(), co_d.data_ptr(), vo_d.data_ptr(),
                                                x_d.data_ptr(), y.data_ptr(), stream)
        assert st == sp.SPMV_OK, sp.spmv_last_error()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(y.cpu().numpy(), oracle.csr_spmv(rp, co, vo, x))


def test_noalloc_rejects_oversized_input(sp):
    lib = sp._lib
    buf = torch.zeros(4, dtype=torch.float64, device="cuda:0")
    p = buf.data_ptr()
    st = lib.spmv_mul_csr_merge_noalloc(1 << 26, 1 << 26, (1 << 26) + 4, p, p, p, p, p, None)
    assert st == sp.SPMV_ERR_UNSUPPORTED
    assert b"exceeds the fixed scratch" in lib.spmv_last_error()
