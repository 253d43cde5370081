"""Python binding of libspmv, the GB300 (sm_103a) SpMV library.

Argument marshalling only: every function calls the C entry point of the same name in
``_build/libspmv.so`` (declared in ``include/spmv.h``) and raises :class:`SpmvError` on
a non-zero status.  Vectors and device arrays are torch CUDA tensors (torch provides
device memory and streams); host arrays may be numpy arrays or CPU tensors.

There is no CPU path: if the compiled library is missing, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libspmv.so")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libspmv.so not built ({LIB_PATH}); run `python -c 'import __graft_entry__ as g; g.build()'`")

_lib = ctypes.CDLL(LIB_PATH)

# ------------------------------------------------------------------ constants (spmv.h)
SPMV_OK, SPMV_ERR_INVALID_ARG, SPMV_ERR_INDEX_RANGE, SPMV_ERR_DUPLICATE, SPMV_ERR_OOM, \
    SPMV_ERR_UNSUPPORTED, SPMV_ERR_CUDA, SPMV_ERR_TIMEOUT, SPMV_ERR_NOT_CONVERTED, SPMV_ERR_IO = range(10)
SPMV_F64, SPMV_F32, SPMV_BF16, SPMV_PATTERN = range(4)
SPMV_FMT_CSR_ROWSPLIT, SPMV_FMT_CSR_MERGE, SPMV_FMT_HB, SPMV_FMT_AUTO, SPMV_FMT_MERGEB = range(5)
SPMV_DEVICE_PTRS = 0x1
SPMV_DUP_SUM = 0x0
SPMV_DUP_ERROR = 0x2
SPMV_INNER_HILBERT, SPMV_INNER_ROWMAJOR, SPMV_INNER_ZMORTON = 0, 1, 2
SPMV_BLOCK_HILBERT, SPMV_BLOCK_ROWMAJOR = 0, 1
SPMV_HB_STAGED, SPMV_HB_CHUNKED = 0, 1
SPMV_COMP_TAU_DEFAULT = 0   # include/spmv.h
SPMV_ACC_DEFAULT, SPMV_ACC_F32, SPMV_ACC_F64, SPMV_ACC_COMPENSATED, SPMV_ACC_SEGMENT = range(5)

FORMATS = {"rowsplit": SPMV_FMT_CSR_ROWSPLIT, "merge": SPMV_FMT_CSR_MERGE, "hb": SPMV_FMT_HB, "auto": SPMV_FMT_AUTO,
           "mergeb": SPMV_FMT_MERGEB}
ELEM_SIZE = {SPMV_F64: 8, SPMV_F32: 4, SPMV_BF16: 2, SPMV_PATTERN: 0}


class spmv_convert_opts(ctypes.Structure):
    _fields_ = [("log2_beta", ctypes.c_int32), ("inner_order", ctypes.c_int32), ("tile", ctypes.c_int32),
                ("hb_product", ctypes.c_int32), ("block_order", ctypes.c_int32)]


class spmv_info_t(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("format", ctypes.c_int32),
                ("dtype", ctypes.c_int32), ("log2_beta", ctypes.c_int32), ("grid_order", ctypes.c_int32),
                ("nblk", ctypes.c_int64), ("merge_tiles", ctypes.c_int64), ("merge_tile_items", ctypes.c_int32),
                ("hb_orders", ctypes.c_int32), ("device_bytes", ctypes.c_int64), ("block_rows", ctypes.c_int64),
                ("mergeb_tiles", ctypes.c_int64)]


class spmv_tune_result(ctypes.Structure):
    _fields_ = [("chosen", ctypes.c_int32), ("reps", ctypes.c_int32), ("ms", ctypes.c_float * 5),
                ("hb_product", ctypes.c_int32), ("pad_", ctypes.c_int32)]


SPMV_TUNE_HB, SPMV_TUNE_MERGEB = 0x1, 0x2


class spmv_server_opts(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_int64), ("slots", ctypes.c_int32), ("max_batch", ctypes.c_int32)]


SPMV_REQ_SPMV, SPMV_REQ_PAGERANK = 0, 1


class spmv_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("matrix", ctypes.c_int32), ("vec_dt", ctypes.c_int32),
                ("accum", ctypes.c_uint32), ("iters", ctypes.c_int32), ("pad_", ctypes.c_int32),
                ("damping", ctypes.c_double), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p)]


class spmv_server_stats_t(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "completed", "failed", "launches", "batched_requests",
                                              "resident_bytes", "peak_bytes", "deferred")]


_p, _i64, _i32, _u32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_uint32
_SIG = {
    "spmv_create_coo": [_i64, _i64, _i64, _p, _p, _p, _i32, _u32, _p, ctypes.POINTER(_p)],
    "spmv_convert": [_p, _i32, ctypes.POINTER(spmv_convert_opts), _p],
    "spmv_mul": [_p, _p, _p, _i32, _u32, _p],
    "spmv_wait": [_p, _p],
    "spmv_mul_batch": [_i32, ctypes.POINTER(_p), _i32, ctypes.POINTER(_p), ctypes.POINTER(_p), _i32, _u32, _p],
    "spmv_destroy": [_p],
    "spmv_info": [_p, ctypes.POINTER(spmv_info_t)],
    "spmv_export_csr": [_p, _p, _p, _p],
    "spmv_export_hb": [_p, _p, _p, _p, _p, _p],
    "spmv_export_merge_partition": [_p, _p, _p],
    "spmv_export_mergeb": [_p, _p, _p, _p],
    "spmv_hilbert_keys": [_i32, _i64, _p, _p, _p, _p],
    "spmv_mul_csr_merge_noalloc": [_i64, _i64, _i64, _p, _p, _p, _p, _p, _p],
    "spmv_pagerank": [_p, ctypes.c_double, _i32, _p, _p],
    "spmv_tune": [_p, _i32, _u32, _u32, ctypes.POINTER(spmv_tune_result), _p],
    "spmv_set_compensation_threshold": [_p, ctypes.c_int64],
    "spmv_save": [_p, ctypes.c_char_p, _p],
    "spmv_cg": [_p, _p, _p, ctypes.c_double, _i32, _p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)],
    "spmv_load": [ctypes.c_char_p, _p, ctypes.POINTER(ctypes.c_void_p)],
    "spmv_server_create": [ctypes.POINTER(spmv_server_opts), ctypes.POINTER(_p)],
    "spmv_server_add": [_p, _p, ctypes.POINTER(ctypes.c_int32)],
    "spmv_server_submit": [_p, ctypes.POINTER(spmv_request), ctypes.POINTER(ctypes.c_int64)],
    "spmv_server_wait": [_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)],
    "spmv_server_replay": [_p, ctypes.c_int64, ctypes.POINTER(spmv_request), _p, _p],
    "spmv_server_stats": [_p, ctypes.POINTER(spmv_server_stats_t)],
    "spmv_server_destroy": [_p],
}
for _name, _args in _SIG.items():
    _f = getattr(_lib, _name)
    _f.argtypes = _args
    _f.restype = ctypes.c_int
_lib.spmv_last_error.restype = ctypes.c_char_p
_lib.spmv_last_error.argtypes = []
_lib.spmv_status_string.restype = ctypes.c_char_p
_lib.spmv_status_string.argtypes = [ctypes.c_int]
_lib.spmv_trace_enable.restype = ctypes.c_int
_lib.spmv_trace_enable.argtypes = [ctypes.c_int]
_lib.spmv_trace_read.restype = ctypes.c_int
_lib.spmv_trace_read.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_char_p), ctypes.POINTER(ctypes.c_longlong),
                                 ctypes.POINTER(ctypes.c_double)]
_lib.spmv_test_fail_alloc.restype = None
_lib.spmv_test_fail_alloc.argtypes = [ctypes.c_longlong]
_lib.spmv_test_wait_timeout.restype = ctypes.c_int
_lib.spmv_test_wait_timeout.argtypes = [ctypes.c_longlong, ctypes.POINTER(ctypes.c_uint32)]


class SpmvError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        msg = _lib.spmv_last_error().decode(errors="replace")
        super().__init__(f"{where}: {_lib.spmv_status_string(status).decode()} {msg}")


def _check(st: int, where: str):
    if st != SPMV_OK:
        raise SpmvError(st, where)


# ------------------------------------------------------------------ marshalling helpers

def _addr(a):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr() or None
    return a.ctypes.data or None


def _is_cuda(a) -> bool:
    return getattr(a, "is_cuda", False)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def dtype_code(a) -> int:
    import torch
    if a is None:
        return SPMV_PATTERN
    t = a.dtype
    if t in (torch.float64, np.float64):
        return SPMV_F64
    if t in (torch.float32, np.float32):
        return SPMV_F32
    if t == torch.bfloat16:
        return SPMV_BF16
    raise TypeError(f"unsupported element type {t}")


class Handle:
    """Owning wrapper of an spmv_handle (destroyed on spmv_destroy or garbage collection)."""

    def __init__(self, ptr: int):
        self.ptr = ptr

    def __del__(self):
        if getattr(self, "ptr", None):
            try:
                _lib.spmv_destroy(self.ptr)
            except Exception:
                pass
            self.ptr = None


# ------------------------------------------------------------------ C ABI, same names

def spmv_create_coo(m, n, row_ind, col_ind, data=None, dtype=None, flags=SPMV_DUP_SUM, stream=None) -> Handle:
    """Ingest triplets (Section 2).  Arrays are all device tensors or all host arrays."""
    nnz = int(row_ind.shape[0])
    dev = _is_cuda(row_ind)
    if dev:
        flags |= SPMV_DEVICE_PTRS
    dt = dtype_code(data) if dtype is None else dtype
    out = ctypes.c_void_p()
    st = _lib.spmv_create_coo(m, n, nnz, _addr(row_ind), _addr(col_ind), _addr(data), dt, flags,
                              _stream(stream), ctypes.byref(out))
    _check(st, "spmv_create_coo")
    return Handle(out.value)


_INNER_DEFAULT = {"csb": SPMV_INNER_ZMORTON, "mergeb": SPMV_INNER_ROWMAJOR, "mergebh": SPMV_INNER_HILBERT}


def spmv_convert(h: Handle, fmt="merge", log2_beta=0, inner_order=None, tile=0,
                 hb_product=SPMV_HB_STAGED, block_order=SPMV_BLOCK_HILBERT, stream=None):
    """Build a storage format (Section 5.1) and make it the active one ("csb": the blocked
    format with row-major block order and Z-Morton inner order, Section 3.1; "mergeb" and
    "mergebh": Merge Blocking with row-wise or Hilbert entries inside the blocks, Section 4.3).
    inner_order None: the format's own inner order (Hilbert for "hb")."""
    if inner_order is None:
        inner_order = _INNER_DEFAULT.get(fmt, SPMV_INNER_HILBERT) if isinstance(fmt, str) else SPMV_INNER_HILBERT
    if fmt == "mergebh":
        fmt = "mergeb"
    if fmt == "csb":
        fmt, block_order = "hb", SPMV_BLOCK_ROWMAJOR
    f = FORMATS[fmt] if isinstance(fmt, str) else int(fmt)
    opts = spmv_convert_opts(log2_beta, inner_order, tile, hb_product, block_order)
    _check(_lib.spmv_convert(h.ptr, f, ctypes.byref(opts), _stream(stream)), "spmv_convert")


def spmv_mul(h: Handle, x, y, accum=SPMV_ACC_DEFAULT, stream=None):
    """y := A x on device tensors x (n) and y (m) of the same dtype (float64 or float32)."""
    vdt = dtype_code(x)
    _check(_lib.spmv_mul(h.ptr, _addr(x), _addr(y), vdt, accum, _stream(stream)), "spmv_mul")
    return y


def spmv_wait(h: Handle, stream=None):
    """Synchronise `stream`; raise SpmvError(SPMV_ERR_TIMEOUT) if a product on h gave up a
    bounded device wait since the last call (see spmv.h)."""
    _check(_lib.spmv_wait(h.ptr, _stream(stream)), "spmv_wait")


def spmv_mul_batch(handles, X, Y, k=1, accum=SPMV_ACC_DEFAULT, stream=None):
    """Y_i := A_i X_i for a list of handles (X_i: n_i x k, Y_i: m_i x k, row-major)."""
    cnt = len(handles)
    hs = (ctypes.c_void_p * cnt)(*[h.ptr for h in handles])
    xs = (ctypes.c_void_p * cnt)(*[_addr(x) for x in X])
    ys = (ctypes.c_void_p * cnt)(*[_addr(y) for y in Y])
    vdt = dtype_code(X[0]) if cnt else SPMV_F64
    _check(_lib.spmv_mul_batch(cnt, hs, k, xs, ys, vdt, accum, _stream(stream)), "spmv_mul_batch")


def spmv_destroy(h: Handle):
    if h.ptr:
        st = _lib.spmv_destroy(h.ptr)
        h.ptr = None
        _check(st, "spmv_destroy")


def spmv_info(h: Handle) -> dict:
    info = spmv_info_t()
    _check(_lib.spmv_info(h.ptr, ctypes.byref(info)), "spmv_info")
    return {name: getattr(info, name) for name, _ in spmv_info_t._fields_ if name != "pad_"}


def spmv_export_csr(h: Handle):
    """(row_ptr, col_ind, data-or-None) as numpy arrays (data in the stored dtype; bf16 as uint16)."""
    inf = spmv_info(h)
    m, nnz, dt = inf["m"], inf["nnz"], inf["dtype"]
    rp = np.empty(m + 1, np.int32)
    co = np.empty(max(nnz, 1), np.int32)
    vals = _host_values(dt, nnz)
    _check(_lib.spmv_export_csr(h.ptr, _addr(rp), _addr(co), _addr(vals)), "spmv_export_csr")
    return rp, co[:nnz], (vals[:nnz] if vals is not None else None)


def spmv_export_hb(h: Handle) -> dict:
    inf = spmv_info(h)
    nnz, nblk, dt = inf["nnz"], inf["nblk"], inf["dtype"]
    idx = np.empty(max(nnz, 1), np.uint32)
    vals = _host_values(dt, nnz)
    bp = np.empty(nblk + 1, np.int32)
    br = np.empty(max(nblk, 1), np.int32)
    bc = np.empty(max(nblk, 1), np.int32)
    _check(_lib.spmv_export_hb(h.ptr, _addr(idx), _addr(vals), _addr(bp), _addr(br), _addr(bc)), "spmv_export_hb")
    return {"idx": idx[:nnz], "val": (vals[:nnz] if vals is not None else None), "blk_ptr": bp,
            "blk_row": br[:nblk], "blk_col": bc[:nblk], "nblk": nblk, "log2beta": inf["log2_beta"]}


def spmv_export_merge_partition(h: Handle):
    tiles = spmv_info(h)["merge_tiles"]
    rs = np.empty(tiles + 1, np.int32)
    ns = np.empty(tiles + 1, np.int32)
    _check(_lib.spmv_export_merge_partition(h.ptr, _addr(rs), _addr(ns)), "spmv_export_merge_partition")
    return rs, ns


def spmv_export_mergeb(h: Handle) -> dict:
    """Merge Blocking tables: the CRS pointer over blocks and every lane's split point (entry and
    block at its first path item), plus the blocked arrays (spmv_export_hb)."""
    inf = spmv_info(h)
    nbr, tiles = inf["block_rows"], inf["mergeb_tiles"]
    rp = np.empty(nbr + 1, np.int32)
    le = np.empty(max(tiles * 32, 1), np.int32)
    lb = np.empty(max(tiles * 32, 1), np.int32)
    _check(_lib.spmv_export_mergeb(h.ptr, _addr(rp), _addr(le), _addr(lb)), "spmv_export_mergeb")
    out = spmv_export_hb(h)
    out.update({"blk_row_ptr": rp, "nbr": nbr, "lane_entry": le[:tiles * 32], "lane_block": lb[:tiles * 32]})
    return out


def spmv_hilbert_keys(K, rows, cols, keys, stream=None):
    """Device Hilbert keys of (rows[i], cols[i]) on the 2^K grid into keys (uint64 as int64 tensor)."""
    _check(_lib.spmv_hilbert_keys(K, int(rows.shape[0]), _addr(rows), _addr(cols), _addr(keys), _stream(stream)),
           "spmv_hilbert_keys")


def spmv_mul_csr_merge_noalloc(m, n, nnz, row_ptr, col_ind, data, x, y, stream=None):
    """y := A x on caller-held device CRS arrays, allocating no device memory (see spmv.h)."""
    _check(_lib.spmv_mul_csr_merge_noalloc(m, n, nnz, _addr(row_ptr), _addr(col_ind), _addr(data), _addr(x),
                                           _addr(y), _stream(stream)), "spmv_mul_csr_merge_noalloc")
    return y


def spmv_pagerank(h: Handle, x, damping=0.85, iters=20, stream=None):
    """PageRank power iteration into the device float64 tensor x (n entries); see spmv.h."""
    _check(_lib.spmv_pagerank(h.ptr, float(damping), int(iters), _addr(x), _stream(stream)), "spmv_pagerank")
    return x


def spmv_trace_enable(on: bool = True):
    """Bracket every library kernel launch with CUDA events (clears the table)."""
    _check(_lib.spmv_trace_enable(1 if on else 0), "spmv_trace_enable")


def spmv_trace_read() -> dict:
    """{kernel name: (launches, total device ms)} of the launches traced so far."""
    cap = 64
    names = (ctypes.c_char_p * cap)()
    counts = (ctypes.c_longlong * cap)()
    ms = (ctypes.c_double * cap)()
    n = _lib.spmv_trace_read(cap, names, counts, ms)
    if n < 0:
        raise SpmvError(SPMV_ERR_CUDA, "spmv_trace_read")
    return {names[i].decode(): (int(counts[i]), float(ms[i])) for i in range(min(n, cap))}


def spmv_last_error() -> str:
    return _lib.spmv_last_error().decode(errors="replace")


def spmv_test_fail_alloc(n: int):
    _lib.spmv_test_fail_alloc(n)


def spmv_test_wait_timeout(polls: int) -> int:
    """Run the bounded-wait check kernel (see spmv.h); returns the status word it wrote."""
    out = ctypes.c_uint32(0)
    _check(_lib.spmv_test_wait_timeout(int(polls), ctypes.byref(out)), "spmv_test_wait_timeout")
    return int(out.value)


def _host_values(dt, nnz):
    if dt == SPMV_F64:
        return np.empty(max(nnz, 1), np.float64)
    if dt == SPMV_F32:
        return np.empty(max(nnz, 1), np.float32)
    if dt == SPMV_BF16:
        return np.empty(max(nnz, 1), np.uint16)
    return None


def spmv_cg(h: Handle, b, x, tol=1e-10, max_iters=1000, stream=None):
    """Conjugate gradients A x = b on device float64 tensors (x overwritten, x0 = 0); returns
    (iterations, final recursive residual norm)."""
    it = ctypes.c_int(0)
    res = ctypes.c_double(0.0)
    _check(_lib.spmv_cg(h.ptr, _addr(b), _addr(x), float(tol), int(max_iters), _stream(stream), ctypes.byref(it),
                        ctypes.byref(res)), "spmv_cg")
    return it.value, res.value


def spmv_save(h: Handle, path: str, stream=None):
    """Write the handle's converted formats to `path` (see spmv.h)."""
    _check(_lib.spmv_save(h.ptr, os.fsencode(path), _stream(stream)), "spmv_save")


def spmv_load(path: str, stream=None) -> Handle:
    """A new handle from a file written by spmv_save (formats restored, no conversion)."""
    out = ctypes.c_void_p()
    _check(_lib.spmv_load(os.fsencode(path), _stream(stream), ctypes.byref(out)), "spmv_load")
    return Handle(out.value)


def spmv_set_compensation_threshold(h: Handle, tau: int):
    """Rows of the row-split product longer than tau are summed with compensation under
    SPMV_ACC_SEGMENT (see spmv.h)."""
    _check(_lib.spmv_set_compensation_threshold(h.ptr, int(tau)), "spmv_set_compensation_threshold")


def spmv_tune(h: Handle, vec_dtype="f64", accum=SPMV_ACC_DEFAULT, hb=False, mergeb=False, stream=None) -> dict:
    """Time one product per storage format and make the fastest the handle's active format."""
    r = spmv_tune_result()
    vdt = SPMV_F64 if vec_dtype in ("f64", SPMV_F64) else SPMV_F32
    flags = (SPMV_TUNE_HB if hb else 0) | (SPMV_TUNE_MERGEB if mergeb else 0)
    _check(_lib.spmv_tune(h.ptr, vdt, accum, flags, ctypes.byref(r), _stream(stream)), "spmv_tune")
    names = {SPMV_FMT_CSR_ROWSPLIT: "rowsplit", SPMV_FMT_CSR_MERGE: "merge", SPMV_FMT_HB: "hb",
             SPMV_FMT_MERGEB: "mergeb"}
    chosen = names[r.chosen]
    if r.chosen == SPMV_FMT_HB and r.hb_product == SPMV_HB_CHUNKED:
        chosen = "hb_chunked"
    ms = dict(zip(["rowsplit", "merge", "hb", "hb_chunked", "mergeb"], [float(v) for v in r.ms]))
    return {"chosen": chosen, "ms": {k: v for k, v in ms.items() if v >= 0}}


class Server:
    """Serving loop (spmv_server_*): resident matrices, admission by slots and memory,
    continuous batching of SpMV requests, PageRank requests."""

    def __init__(self, budget_bytes: int, slots: int = 4, max_batch: int = 64):
        opts = spmv_server_opts(int(budget_bytes), int(slots), int(max_batch))
        out = ctypes.c_void_p()
        _check(_lib.spmv_server_create(ctypes.byref(opts), ctypes.byref(out)), "spmv_server_create")
        self.ptr = out.value

    def add(self, h: Handle) -> int:
        mid = ctypes.c_int32()
        _check(_lib.spmv_server_add(self.ptr, h.ptr, ctypes.byref(mid)), "spmv_server_add")
        return mid.value

    @staticmethod
    def request(kind, matrix, y, x=None, accum=SPMV_ACC_DEFAULT, iters=20, damping=0.85) -> spmv_request:
        vdt = dtype_code(y) if kind == SPMV_REQ_SPMV else SPMV_F64
        return spmv_request(kind, matrix, vdt, accum, iters, 0, damping, _addr(x), _addr(y))

    def submit(self, req: spmv_request) -> int:
        t = ctypes.c_int64()
        _check(_lib.spmv_server_submit(self.ptr, ctypes.byref(req), ctypes.byref(t)), "spmv_server_submit")
        return t.value

    def wait(self, ticket: int) -> float:
        lat = ctypes.c_double()
        _check(_lib.spmv_server_wait(self.ptr, int(ticket), ctypes.byref(lat)), "spmv_server_wait")
        return lat.value

    def replay(self, reqs, arrival_s) -> np.ndarray:
        n = len(reqs)
        arr = (spmv_request * max(n, 1))(*reqs)
        t = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.empty(max(n, 1), np.float64)
        _check(_lib.spmv_server_replay(self.ptr, n, arr, t.ctypes.data, lat.ctypes.data), "spmv_server_replay")
        return lat[:n]

    def stats(self) -> dict:
        st = spmv_server_stats_t()
        _check(_lib.spmv_server_stats(self.ptr, ctypes.byref(st)), "spmv_server_stats")
        return {k: getattr(st, k) for k, _ in spmv_server_stats_t._fields_}

    def close(self):
        if getattr(self, "ptr", None):
            p, self.ptr = self.ptr, None
            _check(_lib.spmv_server_destroy(p), "spmv_server_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def library_path() -> str:
    return LIB_PATH
