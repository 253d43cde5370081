"""Seeded synthetic inputs (sparse patterns, values, vectors) for tests and the benchmark.

Inputs only: nothing here computes a format conversion or a product.  The C
source (``synth.c``) is compiled by :func:`build`; every draw is counter-based
SplitMix64, so results are independent of the thread count.

Workload recipes (stand-ins for the paper's test set, Section 5.2, which is not
available): R-MAT with the Graph500 parameters a/b/c/d = 0.57/0.19/0.19/0.05,
Erdos-Renyi with a fixed number of columns per row, and Zipf power-law rows.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libsynth.so")
_lock = threading.Lock()
_lib = None

RMAT_ABCD = (0.57, 0.19, 0.19, 0.05)


def build(force: bool = False) -> str:
    """Compile synth.c into _build/libsynth.so with gcc (portable flags only)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", src, "-o", tmp, "-lm"])
    os.replace(tmp, _SO)
    return _SO


_GPU_SO = os.path.join(_HERE, "_build", "libsynth_gpu.so")
_gpu = None


def build_gpu(force: bool = False) -> str:
    """Compile synth_gpu.cu (the GPU twin of the R-MAT and value draws) for sm_103a."""
    src = os.path.join(_HERE, "synth_gpu.cu")
    if not force and os.path.exists(_GPU_SO) and os.path.getmtime(_GPU_SO) >= os.path.getmtime(src):
        return _GPU_SO
    os.makedirs(os.path.dirname(_GPU_SO), exist_ok=True)
    tmp = _GPU_SO + f".tmp{os.getpid()}"
    nvcc = os.environ.get("NVCC") or "nvcc"
    if not os.path.exists(nvcc) and os.path.exists("/usr/local/cuda/bin/nvcc"):
        nvcc = "/usr/local/cuda/bin/nvcc"
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-Xcompiler", "-fPIC",
                           "-shared", src, "-o", tmp])
    os.replace(tmp, _GPU_SO)
    return _GPU_SO


def _load_gpu():
    global _gpu
    with _lock:
        if _gpu is None:
            build_gpu()
            lib = ctypes.CDLL(_GPU_SO)
            i64, u64, i32, dbl, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.synth_gpu_rmat.restype = i32
            lib.synth_gpu_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, p, p, p]
            lib.synth_gpu_values.restype = i32
            lib.synth_gpu_values.argtypes = [i64, p, p, u64, i32, i32, p, p]
            _gpu = lib
    return _gpu


def gpu_rmat_raw(scale: int, edge_factor: int = 16, seed: int = 0, abcd=RMAT_ABCD, device="cuda", stream=None):
    """R-MAT edges drawn on the GPU, duplicates kept: (rows, cols) int32 torch tensors on
    `device`, equal to rmat_raw's arrays."""
    import torch
    e = int(edge_factor * (1 << scale))
    rows = torch.empty(e, dtype=torch.int32, device=device)
    cols = torch.empty(e, dtype=torch.int32, device=device)
    a, b, c, _ = abcd
    st = stream if stream is not None else torch.cuda.current_stream(rows.device).cuda_stream
    rc = _load_gpu().synth_gpu_rmat(scale, e, a, b, c, seed, rows.data_ptr(), cols.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"synth_gpu_rmat: CUDA error {rc}")
    return rows, cols


def gpu_values(rows, cols, seed: int = 0, integer: bool = False, f32: bool = False, stream=None):
    """values(rows, cols, seed) computed on the GPU (torch tensors in, a float64 or, with f32,
    float32 tensor out: the doubles rounded to nearest even)."""
    import torch
    out = torch.empty(rows.numel(), dtype=torch.float32 if f32 else torch.float64, device=rows.device)
    st = stream if stream is not None else torch.cuda.current_stream(rows.device).cuda_stream
    rc = _load_gpu().synth_gpu_values(rows.numel(), rows.data_ptr(), cols.data_ptr(), seed, 1 if integer else 0,
                                      1 if f32 else 0, out.data_ptr(), st)
    if rc != 0:
        raise RuntimeError(f"synth_gpu_values: CUDA error {rc}")
    return out


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, u64, i32, dbl, p = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p
            lib.synth_draw.restype = u64
            lib.synth_draw.argtypes = [u64, u64]
            lib.synth_stream_key.restype = u64
            lib.synth_stream_key.argtypes = [u64, u64]
            lib.synth_rmat_raw.restype = None
            lib.synth_rmat_raw.argtypes = [i32, i64, dbl, dbl, dbl, u64, p, p]
            lib.synth_rmat.restype = i64
            lib.synth_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, p, p]
            lib.synth_values.restype = None
            lib.synth_values.argtypes = [i64, p, p, u64, i32, p]
            lib.synth_vector.restype = None
            lib.synth_vector.argtypes = [i64, u64, i32, p]
            lib.synth_er.restype = i64
            lib.synth_er.argtypes = [i64, i32, u64, p, p]
            lib.synth_zipf_lengths.restype = i64
            lib.synth_zipf_lengths.argtypes = [i64, dbl, i64, dbl, u64, p]
            lib.synth_zipf_fill.restype = None
            lib.synth_zipf_fill.argtypes = [i64, u64, p, p, p, p]
            lib.synth_set_threads.restype = None
            lib.synth_set_threads.argtypes = [i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def splitmix_draw(key: int, ctr: int) -> int:
    return int(_load().synth_draw(key, ctr))


def rmat(scale: int, edge_factor: int = 16, seed: int = 0, abcd=RMAT_ABCD, edges: int | None = None):
    """R-MAT pattern on 2^scale vertices, duplicates removed (first occurrence kept).

    Returns (rows, cols) int32 arrays in edge order (unsorted)."""
    lib = _load()
    e = int(edges if edges is not None else edge_factor * (1 << scale))
    rows = np.empty(e, dtype=np.int32)
    cols = np.empty(e, dtype=np.int32)
    a, b, c, _ = abcd
    nnz = lib.synth_rmat(scale, e, a, b, c, seed, _ptr(rows), _ptr(cols))
    if nnz < 0:
        raise MemoryError("synth_rmat: out of host memory")
    return rows[:nnz].copy(), cols[:nnz].copy()


def rmat_raw(scale: int, edge_factor: int = 16, seed: int = 0, abcd=RMAT_ABCD):
    """The R-MAT edges exactly as drawn (duplicates kept, edge order): (rows, cols) int32."""
    lib = _load()
    e = int(edge_factor * (1 << scale))
    rows = np.empty(e, dtype=np.int32)
    cols = np.empty(e, dtype=np.int32)
    a, b, c, _ = abcd
    lib.synth_rmat_raw(scale, e, a, b, c, seed, _ptr(rows), _ptr(cols))
    return rows, cols


def values(rows: np.ndarray, cols: np.ndarray, seed: int = 0, integer: bool = False) -> np.ndarray:
    """Matrix values v(seed, r, c): U[-1,1) doubles, or integers in [-8,8] stored as doubles."""
    lib = _load()
    rows = np.ascontiguousarray(rows, dtype=np.int32)
    cols = np.ascontiguousarray(cols, dtype=np.int32)
    out = np.empty(rows.shape[0], dtype=np.float64)
    lib.synth_values(rows.shape[0], _ptr(rows), _ptr(cols), seed, 1 if integer else 0, _ptr(out))
    return out


def vector(n: int, seed: int = 1, integer: bool = False) -> np.ndarray:
    """Dense vector x_j(seed, j) with the same value kinds as :func:`values`."""
    lib = _load()
    out = np.empty(n, dtype=np.float64)
    lib.synth_vector(n, seed, 1 if integer else 0, _ptr(out))
    return out


def erdos_renyi(n: int, per_row: int = 8, seed: int = 0):
    """n x n pattern with exactly ``per_row`` distinct uniform columns in each row."""
    lib = _load()
    rows = np.empty(n * per_row, dtype=np.int32)
    cols = np.empty(n * per_row, dtype=np.int32)
    if lib.synth_er(n, per_row, seed, _ptr(rows), _ptr(cols)) < 0:
        raise ValueError("per_row > n")
    return rows, cols


def zipf_rows(n: int, alpha: float = 1.8, cap: int = 1 << 20, empty_frac: float = 0.05, seed: int = 0):
    """n x n pattern with Zipf(alpha) row lengths (capped), a fraction of empty rows,
    and distinct uniform columns.  Rows are emitted in row order."""
    lib = _load()
    lens = np.empty(n, dtype=np.int64)
    total = lib.synth_zipf_lengths(n, alpha, min(cap, n), empty_frac, seed, _ptr(lens))
    if total < 0:
        raise MemoryError("synth_zipf_lengths")
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lens, out=off[1:])
    rows = np.empty(total, dtype=np.int32)
    cols = np.empty(total, dtype=np.int32)
    lib.synth_zipf_fill(n, seed, _ptr(off), _ptr(lens), _ptr(rows), _ptr(cols))
    return rows, cols


def shuffle_order(nnz: int, seed: int = 7) -> np.ndarray:
    """A seeded permutation of range(nnz) (to present COO triplets in random order)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.permutation(nnz)


def random_coo(m: int, n: int, nnz: int, seed: int = 0, dup_frac: float = 0.0):
    """Small uniform random COO pattern for unit tests (numpy PCG64; may contain
    duplicates when dup_frac > 0)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    if m == 0 or n == 0:
        return np.zeros(0, np.int32), np.zeros(0, np.int32)
    r = rng.integers(0, m, size=nnz, dtype=np.int64)
    c = rng.integers(0, n, size=nnz, dtype=np.int64)
    key = r * n + c
    _, first = np.unique(key, return_index=True)
    first.sort()
    r, c = r[first], c[first]
    if dup_frac > 0 and r.size > 0:
        k = max(1, int(dup_frac * r.size))
        pick = rng.integers(0, r.size, size=k)
        r = np.concatenate([r, r[pick]])
        c = np.concatenate([c, c[pick]])
        perm = rng.permutation(r.size)
        r, c = r[perm], c[perm]
    return r.astype(np.int32), c.astype(np.int32)


def round_bf16_bits(values: np.ndarray) -> np.ndarray:
    """Input preparation for bfloat16 matrices: each double rounded to the nearest bfloat16
    (ties to even) directly from its 52-bit mantissa, returned as uint16 bit patterns.
    Normal-range values only (zero allowed)."""
    v = np.ascontiguousarray(values, dtype=np.float64)
    b = v.view(np.uint64)
    sign = (b >> np.uint64(63)).astype(np.uint64)
    exp = ((b >> np.uint64(52)) & np.uint64(0x7FF)).astype(np.int64)
    mant = b & np.uint64((1 << 52) - 1)
    q = mant >> np.uint64(45)
    rem = mant & np.uint64((1 << 45) - 1)
    half = np.uint64(1 << 44)
    up = (rem > half) | ((rem == half) & ((q & np.uint64(1)) == np.uint64(1)))
    q = q + up.astype(np.uint64)
    carry = q >> np.uint64(7)
    q = q & np.uint64(0x7F)
    bexp = exp - 1023 + 127 + carry.astype(np.int64)
    zero = (b & np.uint64((1 << 63) - 1)) == 0
    if np.any(~zero & ((bexp < 1) | (bexp > 254))):
        raise ValueError("round_bf16_bits: value outside the normal bfloat16 range")
    out = (sign << np.uint64(15)) | (np.clip(bexp, 0, 255).astype(np.uint64) << np.uint64(7)) | q
    out = np.where(zero, sign << np.uint64(15), out)
    return out.astype(np.uint16)


def bf16_bits_to_float64(bits: np.ndarray) -> np.ndarray:
    return (np.asarray(bits, np.uint16).astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)


def poisson_arrivals(rate: float, n: int, seed: int = 0) -> np.ndarray:
    """n arrival times (seconds from 0) of a Poisson process of `rate` per second."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.cumsum(rng.exponential(1.0 / rate, size=n))


def request_mix(n: int, n_matrices: int, pagerank_frac: float = 0.2, seed: int = 0):
    """(kind, matrix) per request: kind 1 (PageRank) with probability pagerank_frac, else 0
    (SpMV); matrices uniform over range(n_matrices)."""
    rng = np.random.Generator(np.random.PCG64(seed + 1))
    kind = (rng.random(n) < pagerank_frac).astype(np.int32)
    mat = rng.integers(0, n_matrices, size=n).astype(np.int32)
    return kind, mat
