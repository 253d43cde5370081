"""Mixed-precision products (FP32 / bfloat16 / pattern values, FP32 vectors) and PageRank,
through the C ABI, against the FP64 oracle.

Values are rounded once on the host (FP32: IEEE round-to-nearest-even; bfloat16: ties to even
directly from the double, synth.round_bf16_bits); the oracle multiplies the same rounded
values in double precision, so the comparison isolates the accumulation error.  Bounds,
with u = 2^-24 and L the row length:
  FP32 accumulation          |y - ref| <= gamma(L + 1) (|A||x|) + u |ref|
  compensated FP32           |y - ref| <= 8 L u^2 (|A||x|) + u |ref| + 2^-140
  segmented compensation     |y - ref| <= (gamma(8) + 8 L u^2) (|A||x|) + u |ref| + 2^-140
                             (FP32 inside a lane's <= 7 items, TwoSum where lanes and tiles join)
  FP64 accumulation          |y - ref| <= u |ref| + 1e-14 (|A||x|)     (output rounded to FP32)
Integer-valued data with integer x is exact in every mode (all partial sums < 2^24).  The
FP32 bound holds for any order of the additions (the blocked product adds through atomics).
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
U = 2.0 ** -24
DEV = "cuda:0"


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2502_19284_gb300 as sp
    torch.cuda.set_device(0)
    return sp


def store(kind, vals64):
    """(device tensor of stored values or None, the same values as float64 for the oracle)"""
    if kind == "f32":
        v = vals64.astype(np.float32)
        return torch.from_numpy(v).to(DEV), v.astype(np.float64)
    if kind == "bf16":
        bits = synth.round_bf16_bits(vals64)
        t = torch.from_numpy(bits.view(np.int16)).to(DEV).view(torch.bfloat16)
        return t, synth.bf16_bits_to_float64(bits)
    return None, None


def matrices():
    r, c = synth.rmat(14, 16, seed=61)
    yield "rmat14", 1 << 14, r, c
    r, c = synth.zipf_rows(1 << 13, 1.8, 1 << 12, 0.05, seed=62)
    perm = synth.shuffle_order(r.size, 3)
    yield "zipf13", 1 << 13, r[perm], c[perm]


@pytest.mark.parametrize("kind", ["f32", "bf16", "pattern"])
def test_precision_modes(sp, kind):
    for name, n, rows, cols in matrices():
        m = n
        for integer in (False, True):
            vals64 = synth.values(rows, cols, 63, integer=integer)
            vd, v64 = store(kind, vals64)
            x32 = synth.vector(n, 64, integer=integer).astype(np.float32)
            x64 = x32.astype(np.float64)
            rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, v64)
            ref = oracle.csr_spmv(rp, co, vo, x64)
            scale = oracle.csr_absmul(rp, co, vo, x64)
            L = np.diff(rp).astype(np.float64)
            h = sp.spmv_create_coo(m, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV), vd,
                                   dtype=sp.SPMV_PATTERN if vd is None else None)
            xd = torch.from_numpy(x32).to(DEV)
            for algo, modes in (("merge", (sp.SPMV_ACC_F32, sp.SPMV_ACC_COMPENSATED, sp.SPMV_ACC_SEGMENT,
                                           sp.SPMV_ACC_F64)),
                                ("rowsplit", (sp.SPMV_ACC_F32, sp.SPMV_ACC_F64, sp.SPMV_ACC_SEGMENT,
                                              sp.SPMV_ACC_COMPENSATED)),
                                ("hb", (sp.SPMV_ACC_F32, sp.SPMV_ACC_SEGMENT, sp.SPMV_ACC_COMPENSATED))):
                sp.spmv_convert(h, algo)
                for acc in modes:
                    if kind == "pattern" and acc == sp.SPMV_ACC_F64:
                        continue
                    y = torch.full((m,), float("nan"), dtype=torch.float32, device=DEV)
                    sp.spmv_mul(h, xd, y, accum=acc)
                    torch.cuda.synchronize()
                    yg = y.cpu().numpy().astype(np.float64)
                    err = np.abs(yg - ref)
                    if integer:
                        np.testing.assert_array_equal(yg, ref, err_msg=f"{name} {algo} acc{acc}")
                        continue
                    if acc == sp.SPMV_ACC_F32 or algo == "hb":
                        # the blocked product joins a row's runs with FP32 reductions in y, so
                        # its compensated modes keep the FP32 bound (any order of L + 1 roundings)
                        g = (L + 1) * U / (1 - (L + 1) * U)
                        bound = g * scale + U * np.abs(ref)
                    elif acc == sp.SPMV_ACC_COMPENSATED:
                        bound = 8 * L * U * U * scale + U * np.abs(ref) + 2.0 ** -140
                    elif algo == "rowsplit":   # SEGMENT: rows whose class reaches beyond tau compensated
                        g = (L + 1) * U / (1 - (L + 1) * U)
                        cmax = np.array([2, 4, 8, 16, 32, 2048, np.inf])
                        comp = cmax[np.searchsorted(cmax, L)] > sp.SPMV_COMP_TAU_DEFAULT
                        bound = np.where(comp, 8 * L * U * U * scale, g * scale) + U * np.abs(ref) + 2.0 ** -140
                    elif acc == sp.SPMV_ACC_SEGMENT:   # <= 7 FP32 terms per lane, TwoSum joins
                        bound = (8 * U / (1 - 8 * U) + 8 * L * U * U) * scale + U * np.abs(ref) + 2.0 ** -140
                    else:
                        bound = U * np.abs(ref) + 1e-14 * scale
                    assert (err <= bound).all(), (name, algo, acc, float(np.max(err - bound)))


def test_compensation_reduces_error(sp):
    """On long FP32 rows the compensated sum is closer to the exact result than plain FP32."""
    n = 1 << 12
    rows, cols = synth.zipf_rows(n, 1.2, 1 << 12, 0.0, seed=71)
    vals = synth.values(rows, cols, 72).astype(np.float32)
    x32 = synth.vector(n, 73).astype(np.float32)
    rp, co, vo = oracle.coo_to_csr(n, n, rows, cols, vals.astype(np.float64))
    ref = oracle.csr_spmv_neumaier(rp, co, vo, x32.astype(np.float64))
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "merge")
    xd = torch.from_numpy(x32).to(DEV)
    errs = {}
    for acc in (sp.SPMV_ACC_F32, sp.SPMV_ACC_SEGMENT, sp.SPMV_ACC_COMPENSATED):
        y = torch.empty(n, dtype=torch.float32, device=DEV)
        sp.spmv_mul(h, xd, y, accum=acc)
        torch.cuda.synchronize()
        errs[acc] = np.abs(y.cpu().numpy().astype(np.float64) - ref).max()
    assert errs[sp.SPMV_ACC_COMPENSATED] <= errs[sp.SPMV_ACC_SEGMENT] <= errs[sp.SPMV_ACC_F32]


@pytest.mark.parametrize("scale", [10, 14])
def test_pagerank_matches_oracle(sp, scale):
    n = 1 << scale
    rows, cols = synth.rmat(scale, 16, seed=81)
    rp, co, _ = oracle.coo_to_csr(n, n, rows, cols, None)
    ref = oracle.pagerank(rp, co, 0.85, 20)
    for vals in (None, synth.values(rows, cols, 82)):       # stored values are ignored
        h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                               None if vals is None else torch.from_numpy(vals).to(DEV),
                               dtype=sp.SPMV_PATTERN if vals is None else None)
        x = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
        sp.spmv_pagerank(h, x, 0.85, 20)
        torch.cuda.synchronize()
        a = x.cpu().numpy()
        np.testing.assert_allclose(a, ref, rtol=1e-11, atol=1e-16)
        assert abs(a.sum() - 1.0) < 1e-12
        sp.spmv_pagerank(h, x, 0.85, 20)                       # graph replay: same bits
        torch.cuda.synchronize()
        np.testing.assert_array_equal(x.cpu().numpy(), a)
        x2 = torch.empty(n, dtype=torch.float64, device=DEV)
        sp.spmv_pagerank(h, x2, 0.5, 3)                        # new graph for new arguments
        torch.cuda.synchronize()
        np.testing.assert_allclose(x2.cpu().numpy(), oracle.pagerank(rp, co, 0.5, 3), rtol=1e-11, atol=1e-16)


@pytest.mark.parametrize("scale", [12, 17])
def test_pagerank_staged_product_matches_oracle(sp, scale):
    """A handle whose active format is HB (staged product) runs PageRank on the staged blocked
    pattern product: within FP64 rounding of the oracle; a re-conversion that rebuilds the
    staged layout (another block side) drops the captured graph and the result still holds; a
    conversion to the merge path switches back to the bitwise-reproducible product."""
    n = 1 << scale
    rows, cols = synth.rmat(scale, 16, seed=91)
    rp, co, _ = oracle.coo_to_csr(n, n, rows, cols, None)
    ref = oracle.pagerank(rp, co, 0.85, 20)
    vals = synth.values(rows, cols, 92)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    x = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    for lb in (0, 9, 6):
        sp.spmv_convert(h, "hb", log2_beta=lb)
        sp.spmv_pagerank(h, x, 0.85, 20)
        torch.cuda.synchronize()
        a = x.cpu().numpy()
        np.testing.assert_allclose(a, ref, rtol=1e-11, atol=1e-16)
        assert abs(a.sum() - 1.0) < 1e-12
    sp.spmv_convert(h, "merge")
    sp.spmv_pagerank(h, x, 0.85, 20)
    torch.cuda.synchronize()
    b = x.cpu().numpy()
    np.testing.assert_allclose(b, ref, rtol=1e-11, atol=1e-16)
    sp.spmv_pagerank(h, x, 0.85, 20)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(x.cpu().numpy(), b)
    sp.spmv_destroy(h)


def test_compensation_threshold_sweep(sp):
    """Row-split SPMV_ACC_SEGMENT with tau: rows longer than tau (by length class) follow the
    compensated bound, the rest the FP32 bound; tau = 0 equals SPMV_ACC_COMPENSATED bit for
    bit; a negative tau is rejected."""
    n = 1 << 13
    rows, cols = synth.zipf_rows(n, 1.5, 1 << 12, 0.05, seed=75)
    vals = synth.values(rows, cols, 76).astype(np.float32)
    x32 = synth.vector(n, 77).astype(np.float32)
    rp, co, vo = oracle.coo_to_csr(n, n, rows, cols, vals.astype(np.float64))
    x64 = x32.astype(np.float64)
    ref = oracle.csr_spmv(rp, co, vo, x64)
    scale = oracle.csr_absmul(rp, co, vo, x64)
    L = np.diff(rp).astype(np.float64)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, "rowsplit")
    xd = torch.from_numpy(x32).to(DEV)

    def run(acc):
        y = torch.full((n,), float("nan"), dtype=torch.float32, device=DEV)
        sp.spmv_mul(h, xd, y, accum=acc)
        torch.cuda.synchronize()
        return y.cpu().numpy().astype(np.float64)

    comp = run(sp.SPMV_ACC_COMPENSATED)
    cmax = np.array([2, 4, 8, 16, 32, 2048, np.inf])
    cls = np.searchsorted(cmax, L)                 # length class of every row
    for tau in (0, 2, 8, 32, 2048, 1 << 30):
        sp.spmv_set_compensation_threshold(h, tau)
        y = run(sp.SPMV_ACC_SEGMENT)
        compensated = cmax[cls] > tau
        g = (L + 1) * U / (1 - (L + 1) * U)
        bound = np.where(compensated, 8 * L * U * U * scale, g * scale) + U * np.abs(ref) + 2.0 ** -140
        assert (np.abs(y - ref) <= bound).all(), tau
        if tau == 0:
            np.testing.assert_array_equal(y, comp)
    with pytest.raises(sp.SpmvError):
        sp.spmv_set_compensation_threshold(h, -1)
    sp.spmv_destroy(h)
