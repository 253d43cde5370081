"""CPU oracle for the SpMV library -- test infrastructure only.

Plain sequential double-precision restatements of the paper's definitions
(``oracle.c``, compiled with ``-ffp-contract=off``).  Only ``tests/``, the
package's ``smoke()`` check and ``bench.py``'s CPU-baseline leg may import this
module; the library itself never does.

Every function wraps one C routine; the C file's header lists the passage of
the paper each one follows.  Parity pins live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_INDEX_RANGE, ERR_DUPLICATE, ERR_OOM, ERR_UNSUPPORTED = range(6)


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle status {code}")
        self.code = code


def build(force: bool = False, extra_flags: list[str] | None = None, out: str | None = None) -> str:
    """Compile oracle.c with gcc: -O2, floating-point contraction off, portable flags."""
    src = os.path.join(_HERE, "oracle.c")
    so = out or _SO
    if not force and extra_flags is None and os.path.exists(so) and os.path.getmtime(so) >= os.path.getmtime(src):
        return so
    os.makedirs(os.path.dirname(so), exist_ok=True)
    tmp = so + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    cmd += list(extra_flags or []) + [src, "-o", tmp, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, so)
    return so


_PAR_SO = os.path.join(_HERE, "_build", "libparcrs.so")
_par = None


def build_parcrs(force: bool = False) -> str:
    """Compile parcrs.c (the paper's OpenMP row-parallel CRS baseline) with gcc -fopenmp;
    without OpenMP support it is built sequential (parcrs_threads() then reports 1)."""
    src = os.path.join(_HERE, "parcrs.c")
    if not force and os.path.exists(_PAR_SO) and os.path.getmtime(_PAR_SO) >= os.path.getmtime(src):
        return _PAR_SO
    os.makedirs(os.path.dirname(_PAR_SO), exist_ok=True)
    tmp = _PAR_SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    try:
        subprocess.check_call(base + ["-fopenmp", src, "-o", tmp], stderr=subprocess.DEVNULL)
    except subprocess.CalledProcessError:
        subprocess.check_call(base + [src, "-o", tmp])
    os.replace(tmp, _PAR_SO)
    return _PAR_SO


def load_parcrs():
    """Load the ParCRS baseline.  OMP_PROC_BIND defaults to true (Section 5.1); the OpenMP
    runtime reads it when the library is loaded."""
    global _par
    with _lock:
        if _par is None:
            build_parcrs()
            os.environ.setdefault("OMP_PROC_BIND", "true")
            lib = ctypes.CDLL(_PAR_SO)
            lib.parcrs_spmv.restype = None
            lib.parcrs_spmv.argtypes = [ctypes.c_int64] + [ctypes.c_void_p] * 5
            lib.parcrs_threads.restype = ctypes.c_int
            lib.parcrs_threads.argtypes = []
            _par = lib
    return _par


def parcrs_spmv(row_ptr, col, val, x, out=None):
    """y = A x by ParCRS on all host threads (FP64; equal to csr_spmv row for row)."""
    lib = load_parcrs()
    rp, co, vo, xx = _i32(row_ptr), _i32(col), _f64(val), _f64(x)
    m = rp.size - 1
    y = out if out is not None else np.empty(m)
    lib.parcrs_spmv(m, _p(rp), _p(co), _p(vo), _p(xx), _p(y))
    return y


def parcrs_threads():
    return int(load_parcrs().parcrs_threads())


def _declare(lib):
    i64, u64, i32, dbl, p, f32, u16 = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_float, ctypes.c_uint16)
    sig = {
        "oracle_coo_to_csr": (i32, [i64, i64, i64, p, p, p, i32, p, p, p, p]),
        "oracle_csr_spmv": (None, [i64, p, p, p, p, p]),
        "oracle_csr_spmm": (None, [i64, i64, p, p, p, p, p]),
        "oracle_coo_spmv": (None, [i64, i64, p, p, p, p, p]),
        "oracle_csr_spmv_neumaier": (None, [i64, p, p, p, p, p]),
        "oracle_csr_absmul": (None, [i64, p, p, p, p, p]),
        "oracle_csr_transpose": (i32, [i64, i64, p, p, p, p, p, p]),
        "oracle_hilbert_index": (u64, [i32, i64, i64]),
        "oracle_zmorton_index": (u64, [i32, i64, i64]),
        "oracle_grid_order": (i32, [i64, i64]),
        "oracle_log2_beta": (i32, [i64, i64, i64]),
        "oracle_csr_to_hb": (i32, [i64, i64, p, p, p, i32, i32, p, p, p, p, p, p]),
        "oracle_csr_to_csb": (i32, [i64, i64, p, p, p, i32, i32, p, p, p, p, p, p]),
        "oracle_hb_spmv": (None, [i64, i64, i32, p, p, p, p, p, p, p]),
        "oracle_merge_path_walk": (None, [i64, p, i64, p, i64, p, p]),
        "oracle_merge_path_search": (None, [i64, i64, p, i64, p, p]),
        "oracle_merge_spmv": (None, [i64, p, p, p, p, p, i64, p, p]),
        "oracle_block_row_ptr": (None, [i64, p, i64, p]),
        "oracle_mergeb_spmv": (i32, [i64, i64, i32, p, p, p, p, p, p, p, i64]),
        "oracle_round_f32": (f32, [dbl]),
        "oracle_round_bf16": (u16, [dbl]),
        "oracle_bf16_to_double": (dbl, [u16]),
        "oracle_pagerank": (i32, [i64, p, p, dbl, i32, p]),
        "oracle_cg": (i32, [i64, p, p, p, p, dbl, i32, p, p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


def load(path: str | None = None):
    """Load the oracle library (building it first if needed)."""
    global _lib
    if path is not None:
        return _declare(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            build()
            _lib = _declare(ctypes.CDLL(_SO))
    return _lib


def _p(a):
    # the caller keeps `a` referenced until the C call returns (bind converted arrays to a
    # name first: a temporary passed through here would be freed before the call)
    return None if a is None else a.ctypes.data


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


# --------------------------------------------------------------------- wrappers

def coo_to_csr(m, n, rows, cols, vals=None, dup_mode=0, lib=None):
    """Triplet -> CRS (Section 2 / 5.1).  Returns (row_ptr, col_ind, data-or-None)."""
    lib = lib or load()
    rows, cols, vals = _i32(rows), _i32(cols), _f64(vals)
    nnz = rows.shape[0]
    rp = np.empty(m + 1, np.int32)
    co = np.empty(max(nnz, 1), np.int32)
    vo = np.empty(max(nnz, 1), np.float64) if vals is not None else None
    nout = ctypes.c_int64(0)
    st = lib.oracle_coo_to_csr(m, n, nnz, _p(rows), _p(cols), _p(vals), dup_mode, _p(rp), _p(co), _p(vo),
                               ctypes.byref(nout))
    if st != OK:
        raise OracleError(st, "coo_to_csr")
    k = nout.value
    return rp, co[:k].copy(), (vo[:k].copy() if vo is not None else None)


def csr_spmv(row_ptr, col, val, x, lib=None):
    """Algorithm 1."""
    lib = lib or load()
    m = row_ptr.shape[0] - 1
    row_ptr, col, val, x = _i32(row_ptr), _i32(col), _f64(val), _f64(x)
    y = np.empty(m, np.float64)
    lib.oracle_csr_spmv(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y))
    return y


def csr_spmm(row_ptr, col, val, X, lib=None):
    lib = lib or load()
    m = row_ptr.shape[0] - 1
    row_ptr, col, val = _i32(row_ptr), _i32(col), _f64(val)
    X = np.ascontiguousarray(X, np.float64)
    k = X.shape[1]
    Y = np.empty((m, k), np.float64)
    lib.oracle_csr_spmm(m, k, _p(row_ptr), _p(col), _p(val), _p(X), _p(Y))
    return Y


def coo_spmv(m, rows, cols, vals, x, lib=None):
    """Eq. 1 (triplet SpMV)."""
    lib = lib or load()
    rows, cols, vals, x = _i32(rows), _i32(cols), _f64(vals), _f64(x)
    y = np.empty(m, np.float64)
    lib.oracle_coo_spmv(m, rows.shape[0], _p(rows), _p(cols), _p(vals), _p(x), _p(y))
    return y


def csr_spmv_neumaier(row_ptr, col, val, x, lib=None):
    lib = lib or load()
    m = row_ptr.shape[0] - 1
    row_ptr, col, val, x = _i32(row_ptr), _i32(col), _f64(val), _f64(x)
    y = np.empty(m, np.float64)
    lib.oracle_csr_spmv_neumaier(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y))
    return y


def csr_absmul(row_ptr, col, val, x, lib=None):
    """(|A| |x|)_i, the scale in the tolerance |y - y_ref| <= tol * (|A||x|)_i."""
    lib = lib or load()
    m = row_ptr.shape[0] - 1
    row_ptr, col, val, x = _i32(row_ptr), _i32(col), _f64(val), _f64(x)
    y = np.empty(m, np.float64)
    lib.oracle_csr_absmul(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y))
    return y


def csr_transpose(m, n, row_ptr, col, val, lib=None):
    lib = lib or load()
    row_ptr, col, val = _i32(row_ptr), _i32(col), _f64(val)
    nnz = int(row_ptr[m])
    trp = np.empty(n + 1, np.int32)
    tc = np.empty(max(nnz, 1), np.int32)
    tv = np.empty(max(nnz, 1), np.float64) if val is not None else None
    st = lib.oracle_csr_transpose(m, n, _p(row_ptr), _p(col), _p(val), _p(trp), _p(tc), _p(tv))
    if st != OK:
        raise OracleError(st, "csr_transpose")
    return trp, tc[:nnz].copy(), (tv[:nnz].copy() if tv is not None else None)


def hilbert_index(K, r, c, lib=None):
    return int((lib or load()).oracle_hilbert_index(K, r, c))


def hilbert_table(K, lib=None):
    """index[row][col] of the order-K Hilbert curve."""
    lib = lib or load()
    S = 1 << K
    return np.array([[lib.oracle_hilbert_index(K, r, c) for c in range(S)] for r in range(S)], dtype=np.int64)


def zmorton_table(K, lib=None):
    lib = lib or load()
    S = 1 << K
    return np.array([[lib.oracle_zmorton_index(K, r, c) for c in range(S)] for r in range(S)], dtype=np.int64)


def grid_order(m, n, lib=None):
    return int((lib or load()).oracle_grid_order(m, n))


def log2_beta(n, x_bytes=8, slice_budget_bytes=200 * 1024, lib=None):
    """Eq. 2 block size rule with the 16-bit and on-chip slice constraints."""
    return int((lib or load()).oracle_log2_beta(n, x_bytes, slice_budget_bytes))


def csr_to_hb(m, n, row_ptr, col, val, log2beta, inner_order=0, lib=None, block_order=0):
    """CRS -> blocked format: Hilbert block order (block_order 0; inner_order 0 Hilbert, 1
    row-major) or row-major block order (block_order 1, CSB / CSBH; inner_order 0 the block's
    own Hilbert curve, 1 row-major, 2 Z-Morton).  Returns dict of arrays."""
    lib = lib or load()
    row_ptr, col, val = _i32(row_ptr), _i32(col), _f64(val)
    nnz = int(row_ptr[m])
    idx = np.empty(max(nnz, 1), np.uint32)
    vo = np.empty(max(nnz, 1), np.float64) if val is not None else None
    bp = np.empty(nnz + 1, np.int32)
    br = np.empty(max(nnz, 1), np.int32)
    bc = np.empty(max(nnz, 1), np.int32)
    nb = ctypes.c_int64(0)
    fn = lib.oracle_csr_to_csb if block_order == 1 else lib.oracle_csr_to_hb
    st = fn(m, n, _p(row_ptr), _p(col), _p(val), log2beta, inner_order, _p(idx), _p(vo),
            _p(bp), _p(br), _p(bc), ctypes.byref(nb))
    if st != OK:
        raise OracleError(st, "csr_to_hb")
    k = nb.value
    K = grid_order(m, n, lib)
    return {"idx": idx[:nnz].copy(), "val": (vo[:nnz].copy() if vo is not None else None),
            "blk_ptr": bp[:k + 1].copy(), "blk_row": br[:k].copy(), "blk_col": bc[:k].copy(),
            "nblk": k, "log2beta": min(log2beta, K)}


def hb_spmv(m, hb, x, lib=None):
    lib = lib or load()
    bp, br, bc = _i32(hb["blk_ptr"]), _i32(hb["blk_row"]), _i32(hb["blk_col"])
    idx = np.ascontiguousarray(hb["idx"], np.uint32)
    val, x = _f64(hb["val"]), _f64(x)
    y = np.empty(m, np.float64)
    lib.oracle_hb_spmv(m, hb["nblk"], hb["log2beta"], _p(bp), _p(br), _p(bc), _p(idx), _p(val), _p(x), _p(y))
    return y


def merge_path_walk(diag, A, B, lib=None):
    lib = lib or load()
    A = np.ascontiguousarray(A, np.int64)
    B = np.ascontiguousarray(B, np.int64)
    ai, bi = ctypes.c_int64(0), ctypes.c_int64(0)
    lib.oracle_merge_path_walk(diag, _p(A), A.shape[0], _p(B), B.shape[0], ctypes.byref(ai), ctypes.byref(bi))
    return ai.value, bi.value


def merge_path_search(diag, row_ptr, lib=None):
    lib = lib or load()
    row_ptr = _i32(row_ptr)
    m = row_ptr.shape[0] - 1
    ai, bi = ctypes.c_int64(0), ctypes.c_int64(0)
    lib.oracle_merge_path_search(diag, m, _p(row_ptr), int(row_ptr[m]), ctypes.byref(ai), ctypes.byref(bi))
    return ai.value, bi.value


def merge_spmv(row_ptr, col, val, x, parts, lib=None):
    """Merge-based CRS SpMV (Section 3.3) with `parts` sequentially executed parts.
    Returns (y, carry_row, carry_val)."""
    lib = lib or load()
    m = row_ptr.shape[0] - 1
    y = np.empty(m, np.float64)
    cr = np.empty(max(parts, 1), np.int64)
    cv = np.empty(max(parts, 1), np.float64)
    row_ptr, col, val, x = _i32(row_ptr), _i32(col), _f64(val), _f64(x)
    lib.oracle_merge_spmv(m, _p(row_ptr), _p(col), _p(val), _p(x), _p(y), parts, _p(cr), _p(cv))
    return y, cr, cv


def block_row_ptr(blk_row, nblk, nbr, lib=None):
    """CRS pointer over blocks in row-major block order (Section 4.3): nbr + 1 entries."""
    lib = lib or load()
    br = _i32(blk_row)
    ptr = np.empty(nbr + 1, np.int32)
    lib.oracle_block_row_ptr(nblk, _p(br), nbr, _p(ptr))
    return ptr


def csr_to_mergeb(m, n, row_ptr, col, val, log2beta, inner_order=1, lib=None):
    """CRS -> Merge Blocking storage (Section 4.3): the blocks in row-major block order with
    row-wise (inner_order 1, MergeB) or Hilbert (inner_order 0, MergeBH) entries inside, plus
    the block-row pointer (key "blk_row_ptr", nbr = ceil(m / beta) block rows)."""
    lib = lib or load()
    mb = csr_to_hb(m, n, row_ptr, col, val, log2beta, inner_order, lib, block_order=1)
    lb = mb["log2beta"]
    nbr = (m + (1 << lb) - 1) >> lb
    mb["nbr"] = nbr
    mb["blk_row_ptr"] = block_row_ptr(mb["blk_row"], mb["nblk"], nbr, lib)
    return mb


def mergeb_spmv(m, mb, x, parts=1, lib=None):
    """Merge Blocking SpMV (Section 4.3) with `parts` sequentially executed parts."""
    lib = lib or load()
    rp, bp, bc = _i32(mb["blk_row_ptr"]), _i32(mb["blk_ptr"]), _i32(mb["blk_col"])
    idx = np.ascontiguousarray(mb["idx"], np.uint32)
    val, x = _f64(mb["val"]), _f64(x)
    y = np.empty(m, np.float64)
    st = lib.oracle_mergeb_spmv(m, mb["nbr"], mb["log2beta"], _p(rp), _p(bp), _p(bc), _p(idx), _p(val), _p(x),
                                _p(y), parts)
    if st != OK:
        raise OracleError(st, "mergeb_spmv")
    return y


def round_f32(v, lib=None):
    return float((lib or load()).oracle_round_f32(float(v)))


def round_bf16_bits(v, lib=None):
    return int((lib or load()).oracle_round_bf16(float(v)))


def bf16_bits_to_double(b, lib=None):
    return float((lib or load()).oracle_bf16_to_double(int(b)))


def round_array_bf16(a, lib=None):
    """Element-wise RNE double -> bfloat16 (returned as doubles)."""
    lib = lib or load()
    f = lib.oracle_round_bf16
    g = lib.oracle_bf16_to_double
    return np.array([g(f(float(v))) for v in np.asarray(a, np.float64).ravel()], np.float64).reshape(np.shape(a))


def pagerank(row_ptr, col, damping=0.85, iters=20, lib=None):
    lib = lib or load()
    n = row_ptr.shape[0] - 1
    row_ptr, col = _i32(row_ptr), _i32(col)
    x = np.empty(n, np.float64)
    st = lib.oracle_pagerank(n, _p(row_ptr), _p(col), damping, iters, _p(x))
    if st != OK:
        raise OracleError(st, "pagerank")
    return x


def cg(row_ptr, col, val, b, tol=1e-10, max_iters=1000, lib=None):
    """Conjugate gradients from x0 = 0 (see oracle.c).  Returns (x, iterations, ||r||)."""
    lib = lib or load()
    rp, co, vo, bb = _i32(row_ptr), _i32(col), _f64(val), _f64(b)
    n = rp.size - 1
    x = np.empty(n)
    res = ctypes.c_double(0.0)
    it = lib.oracle_cg(n, _p(rp), _p(co), _p(vo), _p(bb), float(tol), int(max_iters), _p(x), ctypes.byref(res))
    if it < 0:
        raise OracleError(ERR_OOM, "oracle_cg")
    return x, it, res.value
