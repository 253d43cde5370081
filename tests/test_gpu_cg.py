"""Conjugate gradients on one resident matrix (spmv_cg), through the C ABI, against the oracle's
CG and against the true residual computed with the oracle's Algorithm 1; every product format."""
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


def spd_rmat(scale, seed):
    """R-MAT B made symmetric positive definite: B + B^T + diag(row sums of |B + B^T| + 1)."""
    r, c = synth.rmat(scale, 8, seed=seed)
    v = synth.values(r, c, seed)
    n = 1 << scale
    rows = np.concatenate([r, c]).astype(np.int32)
    cols = np.concatenate([c, r]).astype(np.int32)
    vals = np.concatenate([v, v])
    d = np.zeros(n)
    np.add.at(d, rows, np.abs(vals))
    rows = np.concatenate([rows, np.arange(n, dtype=np.int32)])
    cols = np.concatenate([cols, np.arange(n, dtype=np.int32)])
    vals = np.concatenate([vals, d + 1.0])
    return n, rows, cols, vals


@pytest.mark.parametrize("fmt", ["merge", "rowsplit", "hb"])
def test_cg_against_oracle(sp, fmt):
    n, rows, cols, vals = spd_rmat(13, 61)
    rp, co, vo = oracle.coo_to_csr(n, n, rows, cols, vals)
    b = synth.vector(n, 62)
    xo, it_o, _ = oracle.cg(rp, co, vo, b, tol=1e-12, max_iters=500)
    h = sp.spmv_create_coo(n, n, torch.from_numpy(rows).to(DEV), torch.from_numpy(cols).to(DEV),
                           torch.from_numpy(vals).to(DEV))
    sp.spmv_convert(h, fmt)
    bd = torch.from_numpy(b).to(DEV)
    x = torch.full((n,), float("nan"), dtype=torch.float64, device=DEV)
    it, res = sp.spmv_cg(h, bd, x, tol=1e-12, max_iters=500)
    xg = x.cpu().numpy()
    if fmt == "hb":
        # the staged product sums runs in no fixed order (double-float products, ~2^-47): at this
        # tolerance CG's iteration count moves with the rounding, so allow 10% more iterations
        assert 0.9 * it_o <= it <= 1.1 * it_o + 8
    else:
        assert it_o <= it <= it_o + 8                # residual read back every 8 iterations
    assert res <= 1e-12 * np.linalg.norm(b) * 10
    true_res = np.linalg.norm(b - oracle.csr_spmv(rp, co, vo, xg))
    assert true_res <= 1e-10 * np.linalg.norm(b)
    assert np.max(np.abs(xg - xo)) <= 1e-9 * np.max(np.abs(xo))
    sp.spmv_destroy(h)


def test_cg_arguments(sp):
    r = np.array([0, 1], np.int32)
    c = np.array([1, 0], np.int32)
    h = sp.spmv_create_coo(2, 3, torch.from_numpy(r).to(DEV), torch.from_numpy(c).to(DEV),
                           torch.ones(2, dtype=torch.float64, device=DEV))
    b = torch.ones(2, dtype=torch.float64, device=DEV)
    x = torch.empty(2, dtype=torch.float64, device=DEV)
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_cg(h, b, x)                           # not converted
    assert e.value.status == sp.SPMV_ERR_NOT_CONVERTED
    sp.spmv_convert(h, "merge")
    with pytest.raises(sp.SpmvError) as e:
        sp.spmv_cg(h, b, x)                           # not square
    assert e.value.status == sp.SPMV_ERR_INVALID_ARG
    sp.spmv_destroy(h)
