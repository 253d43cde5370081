#!/usr/bin/env python
"""Benchmark of the GB300 SpMV library on the R-MAT scale-22 workload.

One step = one pass of the whole hot path over one synthetic matrix:
    ingest the triplets (spmv_create_coo) -> COO->CSR + row-length bins -> row-split SpMV
    -> merge-path partition -> merge-path SpMV (double-float, then native FP64)
    -> CSR->Hilbert-blocked (beta = 2^14) -> blocked SpMV (staged x slices) -> destroy.
Workload: R-MAT scale 22 (4,194,304 rows and columns), edge factor 16, Graph500
a/b/c/d = 0.57/0.19/0.19/0.05, duplicate edges removed, FP64 values and x uniform in
[-1, 1), seeded; the triplets are presented in edge (random) order.  L2 is flushed (a
256 MB write) before every product inside the step, outside the product's events.

value = SpMV GB/s: the compulsory bytes of one FP64 CSR product, nnz (8 + 4) + (m + 1) 4
+ 8 n + 8 m, over the device time of the fastest FP64 spmv_mul call of the step (median
over the timed steps; the call's own kernels only).  The line names that call, carries
every product's time, GB/s, GFLOP/s and error against the oracle, the roofline of that
call's main kernel, the conversions, the whole step, the end-to-end number through host
buffers, clocks sampled during the timed region and the CPU baselines (the oracle on one
core and the paper's ParCRS on all cores, both on the full matrix).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SpMV GB/s vs HBM roofline & GFLOP/s (R-MAT s22); served p50/p99 vs plain FP64"
RMAT = dict(scale=22, edge_factor=16, abcd=(0.57, 0.19, 0.19, 0.05))
FALLBACK_HBM_GBS = 6800.0
FLUSH_BYTES = 256 << 20          # > 2 x the 129 MB L2


# ------------------------------------------------------------------ workload and bytes

def workload_desc(scale):
    return (f"R-MAT scale {scale} (n = 2^{scale}), edge factor 16, a/b/c/d 0.57/0.19/0.19/0.05, deduplicated, "
            "FP64 U(-1,1) values and x, triplets in edge order")


def spmv_bytes(m, n, nnz):
    """Compulsory bytes of one FP64 CSR product (int32 indices): values and columns, row_ptr,
    x read once, y written once."""
    return nnz * 12 + (m + 1) * 4 + n * 8 + m * 8


def row_bytes(m, n, nnz, nblk):
    """Algorithmic bytes of each row of the step, FP64 values, int32 indices."""
    csr = nnz * 12 + (m + 1) * 4
    hb = nnz * 12 + nblk * 12 + 4
    return {
        "ingest": 2 * nnz * 16,                  # read the caller's triplets, write the library copy
        "coo_to_csr": nnz * 16 + csr + (m + 1) * 4 + m * 4,   # triplets in, CSR out; row bins
        "spmv_rowsplit": spmv_bytes(m, n, nnz),
        "merge_partition": 0,                    # O(tiles log m), not part of the compulsory traffic
        "spmv_merge": spmv_bytes(m, n, nnz),
        "spmv_merge_f64": spmv_bytes(m, n, nnz),
        "csr_to_hb": csr + hb,                   # read CSR, write blocked arrays
        "spmv_hb": hb + n * 8 + m * 8,
    }


PRODUCTS = ("spmv_rowsplit", "spmv_merge", "spmv_merge_f64", "spmv_hb")
# the main kernel of each product row (its name in the library's trace and in ncu)
PRODUCT_KERNEL = {"spmv_rowsplit": "k_rowsplit", "spmv_merge": "k_merge_slot_df", "spmv_merge_f64": "k_merge_warp",
                  "spmv_hb": "k_hb_stage"}
PRODUCT_DESC = {"spmv_rowsplit": "row-split CSR (the paper's ParCRS on the GPU), FP64 through double-float",
                "spmv_merge": "merge-path CSR, FP64 through double-float (split FP64 operands, ~2^-47 relative)",
                "spmv_merge_f64": "merge-path CSR, native FP64 arithmetic (SPMV_ACC_F64)",
                "spmv_hb": ("Hilbert-blocked (beta 2^14), block columns with x slices staged in shared memory, "
                            "FP64 through double-float")}


def sort_passes(bits):
    return (bits + 7) // 8


def kernel_bytes(name, m, n, nnz, nblk):
    """Algorithmic bytes that each traced kernel moves in one step (FP64 values, int32
    indices), or None for kernels without a stated figure.  A radix pass reads and writes
    one (64-bit key, 32-bit payload) pair per item: 24 B in the scatter, 8 B (keys) in the
    count.  Sorted items per step: nnz per pass of the COO->CSR sort (row and column bits),
    nnz per pass of the Hilbert-key sort (2K bits), m in the one pass of the row-class sort.
    The product kernels: the compulsory bytes of every launch of the step (one launch
    each, the merge kernels once per accumulation mode)."""
    K = max(1, (max(m, n, 2) - 1).bit_length())
    cbits = max(1, (n - 1).bit_length()) if n > 1 else 1
    rbits = max(1, (m - 1).bit_length()) if m > 1 else 1
    sort_items = (sort_passes(cbits + rbits) + sort_passes(2 * K)) * nnz + m
    table = {
        "k_rs_scatter": 24 * sort_items,
        "k_rs_count": 8 * sort_items,
        "k_gather": 2 * 20 * nnz,                  # perm 4 B + value 8 B read, value 8 B written; twice
        "k_coo_keys": 20 * nnz,                    # row + col read, key + perm written
        "k_hb_keys": 16 * nnz + (m + 1) * 4,       # col read (+ row_ptr), key + perm written
        "k_hb_fill": 16 * nnz,                     # key read, packed index + block head written
        "k_merge_slot_df": spmv_bytes(m, n, nnz),
        "k_merge_warp": spmv_bytes(m, n, nnz),
        "k_rowsplit": spmv_bytes(m, n, nnz),
        "k_hb_spmv": nnz * 12 + nblk * 12 + n * 8 + m * 8,
        "k_hb_stage": nnz * 12 + nblk * 12 + n * 8 + m * 8,
    }
    return table.get(name)


def kernel_units(name, m, n, nnz):
    """Units per step by which a kernel's captured DRAM traffic is scaled to this workload."""
    K = max(1, (max(m, n, 2) - 1).bit_length())
    cbits = max(1, (n - 1).bit_length()) if n > 1 else 1
    rbits = max(1, (m - 1).bit_length()) if m > 1 else 1
    return {"k_rs_scatter": (sort_passes(cbits + rbits) + sort_passes(2 * K)) * nnz + m,
            "k_merge_slot_df": nnz, "k_hb_spmv": nnz, "k_hb_stage": nnz, "k_rowsplit": nnz,
            "k_merge_warp": nnz}.get(name)


def rel_err(y, ref, scale):
    """max_i |y_i - ref_i| / (|A||x|)_i over rows with a nonzero scale (numpy arrays)."""
    import numpy as np
    ok = scale > 0
    if not ok.any():
        return 0.0
    return float(np.max(np.abs(y[ok] - ref[ok]) / scale[ok]))


# ------------------------------------------------------------------ ranks

def max_over_ranks(value, world, dist, device):
    """The largest per-rank time (every rank gets it); the job is as slow as its slowest
    rank.  `device` is the rank's CUDA device (NCCL) or "cpu" (gloo)."""
    if world <= 1:
        return value
    import torch
    t = torch.tensor([value], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(step_bytes, ms_max, world):
    """Whole-job GB/s: every rank processes its own instance of the workload (weak scaling)."""
    return world * step_bytes / (ms_max * 1e-3) / 1e9


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except (OSError, ValueError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [v.strip() for v in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ CPU baselines

class OracleCSR:
    """The oracle's CRS form of the workload (built once, untimed) with Algorithm 1's y and the
    tolerance scale (|A||x|), the reference of every error figure of the line."""

    def __init__(self, m, n, rows, cols, vals, x):
        import oracle
        t = time.perf_counter()
        self.rp, self.co, self.vo = oracle.coo_to_csr(m, n, rows, cols, vals)
        self.coo_to_csr_s = time.perf_counter() - t
        self.m, self.n, self.x = m, n, x
        self.nnz = int(self.co.size)
        self.y = oracle.csr_spmv(self.rp, self.co, self.vo, x)
        self.scale = oracle.csr_absmul(self.rp, self.co, self.vo, x)


def time_min(fn, reps):
    best = None
    for _ in range(reps):
        t = time.perf_counter()
        fn()
        dt = time.perf_counter() - t
        best = dt if best is None else min(best, dt)
    return best


def cpu_baselines(ref, reps_oracle=3, reps_par=10):
    """The oracle's Algorithm 1 on one host core and the paper's ParCRS (Section 5.1: OpenMP
    over rows, dynamic schedule in chunks of 512, threads bound) on every host core, both on
    the full matrix, min of `reps` runs (the paper takes the minimum too).  GB/s of the same
    compulsory bytes as the GPU line."""
    import numpy as np
    import oracle
    b = spmv_bytes(ref.m, ref.n, ref.nnz)
    t1 = time_min(lambda: oracle.csr_spmv(ref.rp, ref.co, ref.vo, ref.x), reps_oracle)
    yp = np.empty(ref.m)
    oracle.parcrs_spmv(ref.rp, ref.co, ref.vo, ref.x, out=yp)      # warm-up (threads, pages)
    tp = time_min(lambda: oracle.parcrs_spmv(ref.rp, ref.co, ref.vo, ref.x, out=yp), reps_par)
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    threads = oracle.parcrs_threads()
    return {
        "value": round(b / t1 / 1e9, 4), "unit": "GB/s", "cores": 1, "kind": "oracle",
        "sample": (f"the full R-MAT scale-22 matrix ({ref.nnz} nonzeros), Algorithm 1 on one core, "
                   f"min of {reps_oracle}: {t1 * 1e3:.1f} ms; the oracle's COO->CSR took {ref.coo_to_csr_s:.2f} s"),
        "parcrs": {"value": round(b / tp / 1e9, 4), "unit": "GB/s", "cores": threads, "host_cores": cores,
                   "ms": round(tp * 1e3, 3), "schedule": "dynamic,512",
                   "omp_proc_bind": os.environ.get("OMP_PROC_BIND"),
                   "equals_oracle": bool(np.array_equal(yp, ref.y)),
                   "kind": "the paper's ParCRS (row-parallel CRS, Section 5.1), FP64, full matrix, min of "
                           f"{reps_par}"},
    }


# ------------------------------------------------------------------ serving leg

SERVE = dict(n_matrices=64, scales=(14, 24), edge_factor=16, budget=150 << 30, slots=8, max_batch=64,
             rates=(1000.0, 5000.0, 10000.0, 20000.0, 50000.0), requests=2000, pagerank_frac=0.2, pagerank_iters=20,
             damping=0.85, check_scale=18, staged_pagerank_scale=22)


def serving_leg(sp, torch, dev, synth, np):
    """Poisson arrivals of SpMV (FP32 values and vectors) and 20-iteration PageRank requests
    on a resident set of R-MAT matrices, through the serving loop, against the same trace on
    the plain one-at-a-time FP64 path (FP64 copies of the matrices, one synchronous call per
    request in arrival order).  Latency = completion - arrival.  Edges are drawn on the GPU
    (synth's twin of the host generator), duplicates summed at ingestion.  Served matrices of
    scale 22 and up are also converted to the staged blocked layout (beta 2^14, active format
    HB): their PageRank requests run on the staged product, their SpMV requests on the batched
    merge path like the others."""
    cfg = SERVE
    rng = np.random.Generator(np.random.PCG64(77))
    scales = rng.integers(cfg["scales"][0], cfg["scales"][1] + 1, size=cfg["n_matrices"])
    h32, h64, xs, ys, prs, x64s, y64s, pr64s, ns = [], [], [], [], [], [], [], [], []
    big = int(np.argmin(np.abs(scales - cfg["check_scale"])))   # the matrix checked against the oracle
    nnz_total = 0
    for i, sc in enumerate(scales):
        n = 1 << int(sc)
        rd, cd = synth.gpu_rmat_raw(int(sc), cfg["edge_factor"], seed=1000 + i, device=dev)
        a = sp.spmv_create_coo(n, n, rd, cd, synth.gpu_values(rd, cd, seed=1000 + i, f32=True))
        sp.spmv_convert(a, "merge")
        if sc >= cfg["staged_pagerank_scale"]:   # PageRank on the staged blocked product
            sp.spmv_convert(a, "hb", log2_beta=14)
        b = sp.spmv_create_coo(n, n, rd, cd, synth.gpu_values(rd, cd, seed=1000 + i))
        sp.spmv_convert(b, "auto")
        del rd, cd
        nnz_total += sp.spmv_info(a)["nnz"]
        h32.append(a)
        h64.append(b)
        x = synth.vector(n, seed=2000 + i)
        xs.append(torch.from_numpy(x.astype(np.float32)).pin_memory())
        ys.append(torch.empty(n, dtype=torch.float32).pin_memory())
        prs.append(torch.empty(n, dtype=torch.float64).pin_memory())
        x64s.append(torch.from_numpy(x).pin_memory())
        y64s.append(torch.empty(n, dtype=torch.float64).pin_memory())
        pr64s.append(torch.empty(n, dtype=torch.float64, device=dev))
        ns.append(n)
    torch.cuda.synchronize()
    srv = sp.Server(cfg["budget"], slots=cfg["slots"], max_batch=cfg["max_batch"])
    ids = [srv.add(h) for h in h32]
    dx = [torch.empty(n, dtype=torch.float64, device=dev) for n in ns]
    dy = [torch.empty(n, dtype=torch.float64, device=dev) for n in ns]
    out = {"config": {"matrices": int(cfg["n_matrices"]), "scales": [int(v) for v in scales],
                      "nnz": int(nnz_total), "edge_factor": cfg["edge_factor"],
                      "values": "f32 (served) / f64 (plain); duplicate edges summed",
                      "mix": f"{1 - cfg['pagerank_frac']:.0%} SpMV / {cfg['pagerank_frac']:.0%} PageRank-"
                             f"{cfg['pagerank_iters']}", "budget_bytes": cfg["budget"], "slots": cfg["slots"],
                      "max_batch": cfg["max_batch"], "requests_per_rate": cfg["requests"],
                      "pagerank_product": (f"staged blocked (HB, beta 2^14) for scales >= {cfg['staged_pagerank_scale']}, "
                                           "merge path below"),
                      "resident_bytes": srv.stats()["resident_bytes"]},
           "rates": []}
    # accuracy of a served FP32 product against the oracle (the matrix of scale closest to
    # check_scale): Algorithm 1 in FP64 on the FP32-rounded triplet values and FP32 x
    # (accumulation error; the library also sums duplicate triplets in FP32) and on the
    # original FP64 values and x (total error), both as max_i |y_i - ref_i| / (|A||x|)_i
    import oracle
    t = srv.submit(sp.Server.request(sp.SPMV_REQ_SPMV, ids[big], ys[big], x=xs[big]))
    srv.wait(t)
    a_ = ys[big].numpy().astype(np.float64)
    br, bc = synth.rmat_raw(int(scales[big]), cfg["edge_factor"], seed=1000 + big)
    bv = synth.values(br, bc, seed=1000 + big)
    nb = ns[big]
    rp, co, vo = oracle.coo_to_csr(nb, nb, br, bc, bv)
    _, _, vo32 = oracle.coo_to_csr(nb, nb, br, bc, bv.astype(np.float32).astype(np.float64))
    x64 = x64s[big].numpy()
    x32r = xs[big].numpy().astype(np.float64)
    out["accuracy"] = {
        "reference": "oracle (Algorithm 1, FP64)",
        "max_accumulation_err": rel_err(a_, oracle.csr_spmv(rp, co, vo32, x32r), oracle.csr_absmul(rp, co, vo32, x32r)),
        "max_total_err": rel_err(a_, oracle.csr_spmv(rp, co, vo, x64), oracle.csr_absmul(rp, co, vo, x64)),
        "matrix_scale": int(scales[big])}
    del rp, co, vo, vo32
    # service time of every request kind and matrix alone (device events, FP32 handles): the
    # bound on throughput for a trace served one request at a time with the GPU to itself
    ev = lambda: torch.cuda.Event(enable_timing=True)
    t_spmv, t_pr = [], []
    for i, h in enumerate(h32):
        xd = xs[i].to(dev)
        yd = torch.empty(ns[i], dtype=torch.float32, device=dev)
        prd = torch.empty(ns[i], dtype=torch.float64, device=dev)
        sp.spmv_mul(h, xd, yd)
        sp.spmv_pagerank(h, prd, cfg["damping"], cfg["pagerank_iters"])
        e = [ev() for _ in range(3)]
        e[0].record()
        sp.spmv_mul(h, xd, yd)
        e[1].record()
        sp.spmv_pagerank(h, prd, cfg["damping"], cfg["pagerank_iters"])
        e[2].record()
        torch.cuda.synchronize()
        t_spmv.append(e[0].elapsed_time(e[1]))
        t_pr.append(e[1].elapsed_time(e[2]))
        del xd, yd, prd
    out["service_ms_alone"] = {"spmv_mean": round(float(np.mean(t_spmv)), 4), "pagerank_mean": round(float(np.mean(t_pr)), 3),
                               "spmv_max": round(float(np.max(t_spmv)), 4), "pagerank_max": round(float(np.max(t_pr)), 3)}
    for rate in cfg["rates"]:
        N = cfg["requests"]
        kind, mat = synth.request_mix(N, len(ns), cfg["pagerank_frac"], seed=int(rate))
        arr = synth.poisson_arrivals(rate, N, seed=int(rate))
        busy_ms = float(sum(t_pr[m] if k == 1 else t_spmv[m] for k, m in zip(kind, mat)))
        reqs = []
        for k, m in zip(kind, mat):
            if k == 1:
                reqs.append(sp.Server.request(sp.SPMV_REQ_PAGERANK, ids[m], prs[m], iters=cfg["pagerank_iters"],
                                              damping=cfg["damping"]))
            else:
                reqs.append(sp.Server.request(sp.SPMV_REQ_SPMV, ids[m], ys[m], x=xs[m]))
        st0 = srv.stats()
        t0 = time.perf_counter()
        lat = srv.replay(reqs, arr)
        wall = time.perf_counter() - t0
        st1 = srv.stats()
        served = {"p50_ms": round(float(np.percentile(lat, 50)) * 1e3, 3),
                  "p99_ms": round(float(np.percentile(lat, 99)) * 1e3, 3),
                  "throughput_rps": round(N / float(np.max(arr + lat)), 1),
                  "launches": st1["launches"] - st0["launches"],
                  "batched_spmv": st1["batched_requests"] - st0["batched_requests"],
                  "deferred": st1["deferred"] - st0["deferred"], "wall_s": round(wall, 3)}
        # plain path: one request at a time, FP64, synchronous, in arrival order
        plat = np.empty(N)
        start = time.perf_counter() + 1e-3
        stream = torch.cuda.current_stream()
        for i, (k, m) in enumerate(zip(kind, mat)):
            ta = start + arr[i]
            while time.perf_counter() < ta:
                pass
            if k == 1:
                sp.spmv_pagerank(h64[m], pr64s[m], cfg["damping"], cfg["pagerank_iters"])
                prs[m].copy_(pr64s[m], non_blocking=True)
            else:
                dx[m].copy_(x64s[m], non_blocking=True)
                sp.spmv_mul(h64[m], dx[m], dy[m])
                y64s[m].copy_(dy[m], non_blocking=True)
            stream.synchronize()
            plat[i] = time.perf_counter() - ta
        plain = {"p50_ms": round(float(np.percentile(plat, 50)) * 1e3, 3),
                 "p99_ms": round(float(np.percentile(plat, 99)) * 1e3, 3),
                 "throughput_rps": round(N / float(np.max(arr + plat)), 1)}
        out["rates"].append({"rate_rps": rate, "served": served, "plain_fp64": plain,
                             "one_at_a_time_capacity_rps": round(N / (busy_ms * 1e-3), 1)})
    srv.close()
    for h in h32 + h64:
        sp.spmv_destroy(h)
    return out


# ------------------------------------------------------------------ batched leg

BATCH = dict(n_matrices=512, scales=(10, 20), edge_factors=(8, 32), ks=(1, 4, 16), reps=3, oracle_checks=6)
BATCH_SMALL = dict(n_matrices=64, scales=(10, 18), edge_factors=(8, 32), ks=(1, 4, 16), reps=5, oracle_checks=6)


def batched_leg(sp, torch, dev, synth, np, cfg):
    """Many R-MAT matrices of uneven size (FP32 values) times k FP32 right-hand sides in one
    captured batched launch (spmv_mul_batch), against the plain path: one FP64 spmv_mul per
    matrix and right-hand side.  Edges are drawn on the GPU (synth's GPU twin of the host
    generator) and ingested with duplicates summed.  Before the k = 1 batch the autotuner
    times every format and product per matrix and keeps the fastest (row-split, merge-path,
    staged blocked, chunked blocked); k > 1 batches run on the merge-path tiles.  A sample of
    matrices is checked against the oracle.  GFLOP/s = 2 nnz k / time (device events)."""
    import oracle
    rng = np.random.Generator(np.random.PCG64(88))
    scales = rng.integers(cfg["scales"][0], cfg["scales"][1] + 1, size=cfg["n_matrices"])
    efs = rng.integers(cfg["edge_factors"][0], cfg["edge_factors"][1] + 1, size=cfg["n_matrices"])
    h32, h64, ns, nnz_total, edges_total = [], [], [], 0, 0
    t0 = time.perf_counter()
    for i, (sc, ef) in enumerate(zip(scales, efs)):
        n = 1 << int(sc)
        rd, cd = synth.gpu_rmat_raw(int(sc), int(ef), seed=5000 + i, device=dev)
        a = sp.spmv_create_coo(n, n, rd, cd, synth.gpu_values(rd, cd, seed=5000 + i, f32=True))
        sp.spmv_convert(a, "merge")
        b = sp.spmv_create_coo(n, n, rd, cd, synth.gpu_values(rd, cd, seed=5000 + i))
        sp.spmv_convert(b, "merge")
        del rd, cd
        h32.append(a)
        h64.append(b)
        ns.append(n)
        nnz_total += sp.spmv_info(a)["nnz"]
        edges_total += int(ef) << int(sc)
    build_s = time.perf_counter() - t0
    ev = lambda: torch.cuda.Event(enable_timing=True)

    def time_batch(k, X, Y, reps):
        sp.spmv_mul_batch(h32, X, Y, k=k, accum=sp.SPMV_ACC_F32)          # plan + graph capture
        torch.cuda.synchronize()
        a_, b_ = ev(), ev()
        a_.record()
        for _ in range(reps):
            sp.spmv_mul_batch(h32, X, Y, k=k, accum=sp.SPMV_ACC_F32)
        b_.record()
        torch.cuda.synchronize()
        return a_.elapsed_time(b_) / reps

    X1 = [torch.randn(n, 1, dtype=torch.float32, device=dev) for n in ns]
    Y1 = [torch.empty(n, 1, dtype=torch.float32, device=dev) for n in ns]
    ms_untuned = time_batch(1, X1, Y1, cfg["reps"])     # every matrix on the merge-path tiles
    del X1, Y1
    t0 = time.perf_counter()
    choice = {}
    for h in h32:
        res = sp.spmv_tune(h, "f32", accum=sp.SPMV_ACC_F32, hb=True)
        choice[res["chosen"]] = choice.get(res["chosen"], 0) + 1
    tune_s = time.perf_counter() - t0
    out = {"config": {"matrices": int(cfg["n_matrices"]), "scales": [int(cfg["scales"][0]), int(cfg["scales"][1])],
                      "edge_factors": [int(cfg["edge_factors"][0]), int(cfg["edge_factors"][1])],
                      "edges": int(edges_total), "nnz": int(nnz_total),
                      "values": "f32 batched / f64 plain (duplicate edges summed)", "rhs": "f32 batched / f64 plain",
                      "generate_convert_s": round(build_s, 2), "tune_s": round(tune_s, 2)},
           "autotuner_choice": choice,
           "k1_all_merge_ms": round(ms_untuned, 4),
           "k1_all_merge_gflops": round(2.0 * nnz_total / ms_untuned / 1e6, 1), "k": []}
    checked = []
    t0, t1 = ev(), ev()
    for k in cfg["ks"]:
        X = [torch.randn(n, k, dtype=torch.float32, device=dev) for n in ns]
        Y = [torch.empty(n, k, dtype=torch.float32, device=dev) for n in ns]
        ms_b = time_batch(k, X, Y, cfg["reps"])
        if k == 1:   # oracle check of a sample of matrices (evenly spaced over the batch)
            for i in np.linspace(0, len(ns) - 1, cfg["oracle_checks"]).astype(int).tolist():
                n = ns[i]
                rr, cc = synth.rmat_raw(int(scales[i]), int(efs[i]), seed=5000 + i)
                vv = synth.values(rr, cc, seed=5000 + i).astype(np.float32).astype(np.float64)
                rp, co, vo = oracle.coo_to_csr(n, n, rr, cc, vv)
                xr = X[i][:, 0].double().cpu().numpy()
                yr = oracle.csr_spmv(rp, co, vo, xr)
                sc_ = oracle.csr_absmul(rp, co, vo, xr)
                checked.append({"matrix": i, "scale": int(scales[i]), "nnz": int(co.size),
                                "max_err": rel_err(Y[i][:, 0].double().cpu().numpy(), yr, sc_)})
        # plain: one FP64 product per matrix and column
        X64 = [x.double() for x in X]
        cols = [[x[:, q].contiguous() for q in range(k)] for x in X64]
        y64 = [torch.empty(n, dtype=torch.float64, device=dev) for n in ns]
        for h, cs, y in zip(h64, cols, y64):
            sp.spmv_mul(h, cs[0], y)
        torch.cuda.synchronize()
        t0.record()
        for h, cs, y in zip(h64, cols, y64):
            for xc in cs:
                sp.spmv_mul(h, xc, y)
        t1.record()
        torch.cuda.synchronize()
        ms_p = t0.elapsed_time(t1)
        flops = 2.0 * nnz_total * k
        out["k"].append({"k": k, "batched_ms": round(ms_b, 4), "batched_gflops": round(flops / ms_b / 1e6, 1),
                         "plain_fp64_ms": round(ms_p, 4), "plain_fp64_gflops": round(flops / ms_p / 1e6, 1),
                         "speedup": round(ms_p / ms_b, 2)})
        del X, Y, X64, cols, y64
    out["oracle_checks"] = {"reference": "oracle (Algorithm 1, FP64) on the FP32-rounded values, k = 1",
                            "accumulation": "f32", "matrices": checked}
    for h in h32 + h64:
        sp.spmv_destroy(h)
    torch.cuda.synchronize()
    return out


# ------------------------------------------------------------------ iterative leg

def iterative_leg(sp, torch, dev, synth, np):
    """Conjugate gradients on one resident matrix: B + B^T + diag(row sums of |B + B^T| + 1)
    from R-MAT scale 20 (edge factor 8, FP64, symmetric positive definite), solved to 1e-6 in
    the merge-path and in the staged blocked format (tolerance 1e-6).  Reports the conversion, the solve, the
    iterations and the conversion amortised over them (Sections 6.2 and 7), and for the blocked
    format the time to load the converted matrix from disk instead (spmv_save / spmv_load)."""
    import tempfile
    scale, ef, seed = 20, 8, 4242
    n = 1 << scale
    r, c = synth.gpu_rmat_raw(scale, ef, seed=seed, device=dev)
    v = synth.gpu_values(r, c, seed=seed)
    rows = torch.cat([r, c, torch.arange(n, dtype=torch.int32, device=dev)])
    cols = torch.cat([c, r, torch.arange(n, dtype=torch.int32, device=dev)])
    d = torch.zeros(n, dtype=torch.float64, device=dev)
    d.index_add_(0, torch.cat([r, c]).long(), torch.cat([v, v]).abs())
    vals = torch.cat([v, v, d + 1.0])
    del r, c, v, d
    b = torch.from_numpy(synth.vector(n, seed + 1)).to(dev)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"matrix": f"R-MAT scale {scale}, edge factor {ef}, made SPD (B + B^T + diagonal), FP64",
           "tol": 1e-6, "formats": []}
    for fmt in ("merge", "hb"):
        torch.cuda.synchronize()
        e = [ev() for _ in range(4)]
        e[0].record()
        h = sp.spmv_create_coo(n, n, rows, cols, vals)
        e[1].record()
        sp.spmv_convert(h, fmt)
        e[2].record()
        it, res = sp.spmv_cg(h, b, x, tol=1e-6, max_iters=500)
        e[3].record()
        torch.cuda.synchronize()
        y = torch.empty(n, dtype=torch.float64, device=dev)
        p0, p1 = ev(), ev()
        p0.record()
        for _ in range(10):
            sp.spmv_mul(h, b, y)
        p1.record()
        torch.cuda.synchronize()
        conv = e[0].elapsed_time(e[2])
        solve = e[2].elapsed_time(e[3])
        entry = {"format": fmt, "nnz": sp.spmv_info(h)["nnz"], "convert_ms": round(conv, 3),
                 "cg_iterations": it, "cg_residual": res, "solve_ms": round(solve, 3),
                 "ms_per_iteration": round(solve / max(it, 1), 4), "product_ms": round(p0.elapsed_time(p1) / 10, 4),
                 "convert_per_iteration_ms": round(conv / max(it, 1), 4)}
        if fmt == "hb":
            with tempfile.TemporaryDirectory() as tmp:
                path = os.path.join(tmp, "a.spmv")
                t0 = time.perf_counter()
                sp.spmv_save(h, path)
                t1 = time.perf_counter()
                g = sp.spmv_load(path)
                torch.cuda.synchronize()
                t2 = time.perf_counter()
                entry.update(save_s=round(t1 - t0, 3), load_s=round(t2 - t1, 3),
                             file_bytes=os.path.getsize(path))
                sp.spmv_destroy(g)
        out["formats"].append(entry)
        sp.spmv_destroy(h)
    return out


# ------------------------------------------------------------------ Merge Blocking leg

def blocking_leg(sp, torch, dev, m, n, r_d, c_d, v_d, x_d, flush, traffic_db, reps=10):
    """Merge Blocking (Section 4.3) on the step's workload, outside the timed step: the
    conversion CSR -> MergeB (row-wise inside blocks) and CSR -> MergeBH (Hilbert inside
    blocks) at beta = 2^14, each a full rebuild from the CRS arrays (median of 3), and each
    product (L2 flushed before every call; median of `reps`), with its main kernel's device
    time from the library's trace against the blocked format's compulsory bytes.  Returns the
    figures and the two products' y for the oracle errors."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    h = sp.spmv_create_coo(m, n, r_d, c_d, v_d)
    sp.spmv_convert(h, "rowsplit")
    out, ys = {}, {}
    conv = {"mergeb": [], "mergebh": []}
    for _ in range(3):
        for fmt in ("mergeb", "mergebh"):
            torch.cuda.synchronize()
            e0, e1 = ev(), ev()
            e0.record()
            sp.spmv_convert(h, fmt, log2_beta=14)
            e1.record()
            torch.cuda.synchronize()
            conv[fmt].append(e0.elapsed_time(e1))
    for fmt in ("mergeb", "mergebh"):
        sp.spmv_convert(h, fmt, log2_beta=14)
        info = sp.spmv_info(h)
        nnz, nblk = info["nnz"], info["nblk"]
        y = torch.empty(m, dtype=torch.float64, device=dev)
        for _ in range(3):
            sp.spmv_mul(h, x_d, y)
        torch.cuda.synchronize()
        sp.spmv_trace_enable(True)
        t = []
        for _ in range(reps):
            flush.fill_(1)
            e0, e1 = ev(), ev()
            e0.record()
            sp.spmv_mul(h, x_d, y)
            e1.record()
            t.append((e0, e1))
        torch.cuda.synchronize()
        trace = sp.spmv_trace_read()
        sp.spmv_trace_enable(False)
        ms = statistics.median(a.elapsed_time(b) for a, b in t)
        kb = nnz * 12 + nblk * 12 + n * 8 + m * 8
        cnt, kms = trace.get("k_mergeb", (0, 0.0))
        kdur = kms / cnt if cnt else None
        t = traffic_db.get("k_mergeb")
        traffic = None
        if fmt == "mergeb" and t and t.get("source_sha") == source_sha(t.get("source"), t.get("from"), t.get("to")):
            traffic = int(t["bytes_per_unit"] * nnz)   # ncu DRAM bytes (scale 21, MergeB) scaled to one launch
        out[fmt] = {"convert_ms": round(statistics.median(conv[fmt]), 3), "product_ms": round(ms, 4),
                    "kernel_traffic": traffic,
                    "gbs": round(kb / (ms * 1e-3) / 1e9, 1), "gflops": round(2 * nnz / (ms * 1e-3) / 1e9, 1),
                    "kernel_ms": None if kdur is None else round(kdur, 4),
                    "kernel_gbs": None if kdur is None else round(kb / (kdur * 1e-3) / 1e9, 1),
                    "compulsory_bytes": kb, "nblk": nblk, "block_rows": info["block_rows"],
                    "warp_tiles": info["mergeb_tiles"]}
        ys[fmt] = y
    sp.spmv_destroy(h)
    out["what"] = ("Merge Blocking at beta 2^14: merge path over (block-row ends, entries) in warp tiles of 256 "
                   "items, run sums reduced into y; native FP64 accumulation")
    return out, ys


# ------------------------------------------------------------------ precision leg

def precision_leg(sp, torch, dev, synth, np):
    """Stored values FP64 / FP32 / BF16 / pattern times each accumulation mode on two matrices
    (Erdos-Renyi n = 2^23 with 8 per row; Zipf(1.8) rows on n = 2^22, capped at 2^20, 5% empty).
    Errors against the oracle (Algorithm 1 in FP64), max_i |y_i - ref_i| / (|A||x|)_i:
    'accumulation' on the same rounded values and x, 'total' on the original FP64 values and x."""
    import oracle

    def mats():
        n = 1 << 23
        r, c = synth.erdos_renyi(n, 8, seed=11)
        yield "erdos_renyi n=2^23 8/row", n, r, c
        n = 1 << 22
        r, c = synth.zipf_rows(n, 1.8, 1 << 20, 0.05, seed=12)
        yield "zipf(1.8) rows n=2^22 cap 2^20 5% empty", n, r, c
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = []
    for name, n, r, c in mats():
        v64 = synth.values(r, c, seed=13)
        x64 = synth.vector(n, seed=14)
        x32r = x64.astype(np.float32).astype(np.float64)     # the FP32 x as exact doubles
        rd, cd = torch.from_numpy(r).to(dev), torch.from_numpy(c).to(dev)
        xd64 = torch.from_numpy(x64).to(dev)
        xd32 = xd64.float()
        rp, co, vo = oracle.coo_to_csr(n, n, r, c, v64)
        y_exact = oracle.csr_spmv(rp, co, vo, x64)
        s_exact = oracle.csr_absmul(rp, co, vo, x64)
        v64d = torch.from_numpy(v64).to(dev)
        entry = {"matrix": name, "n": n, "nnz": int(r.size), "reference": "oracle (Algorithm 1, FP64)", "modes": []}
        for kind in ("f64", "f32", "bf16", "pattern"):
            if kind == "f64":
                vstore, vr = v64d, vo
            elif kind == "f32":
                vstore, vr = v64d.float(), vo.astype(np.float32).astype(np.float64)
            elif kind == "bf16":
                bits = synth.round_bf16_bits(v64)
                vstore = torch.from_numpy(bits.view(np.int16)).to(dev).view(torch.bfloat16)
                vr = synth.bf16_bits_to_float64(synth.round_bf16_bits(vo))
            else:
                vstore, vr = None, None
            xin = xd64 if kind == "f64" else xd32
            xref = x64 if kind == "f64" else x32r
            y_ref = oracle.csr_spmv(rp, co, vr, xref)
            s_ref = oracle.csr_absmul(rp, co, vr, xref)
            h = sp.spmv_create_coo(n, n, rd, cd, vstore, dtype=sp.SPMV_PATTERN if vstore is None else None)
            sp.spmv_convert(h, "merge")
            modes = ([("default (double-float)", sp.SPMV_ACC_DEFAULT), ("f64", sp.SPMV_ACC_F64)] if kind == "f64" else
                     [("f32", sp.SPMV_ACC_F32), ("segment", sp.SPMV_ACC_SEGMENT),
                      ("compensated", sp.SPMV_ACC_COMPENSATED)] + ([("f64", sp.SPMV_ACC_F64)] if kind != "pattern" else []))
            y = torch.empty(n, dtype=xin.dtype, device=dev)
            for mname, acc in modes:
                sp.spmv_mul(h, xin, y, accum=acc)
                torch.cuda.synchronize()
                t0, t1 = ev(), ev()
                t0.record()
                for _ in range(5):
                    sp.spmv_mul(h, xin, y, accum=acc)
                t1.record()
                torch.cuda.synchronize()
                ms = t0.elapsed_time(t1) / 5
                yh = y.double().cpu().numpy()
                es = {"f64": 8, "f32": 4, "bf16": 2, "pattern": 0}[kind]
                xs = 8 if kind == "f64" else 4
                nbytes = r.size * (4 + es) + (n + 1) * 4 + 2 * n * xs
                entry["modes"].append({"values": kind, "accumulation": mname, "ms": round(ms, 4),
                                       "gbs": round(nbytes / ms / 1e6, 1), "gflops": round(2 * r.size / ms / 1e6, 1),
                                       "max_accumulation_err": rel_err(yh, y_ref, s_ref),
                                       "max_total_err": None if kind == "pattern" else rel_err(yh, y_exact, s_exact)})
            if kind == "f32":   # compensation threshold tau of the row-split product
                sp.spmv_convert(h, "rowsplit")
                sweep = []
                for tau in TAUS:
                    sp.spmv_set_compensation_threshold(h, tau)
                    sp.spmv_mul(h, xin, y, accum=sp.SPMV_ACC_SEGMENT)
                    torch.cuda.synchronize()
                    t0, t1 = ev(), ev()
                    t0.record()
                    for _ in range(5):
                        sp.spmv_mul(h, xin, y, accum=sp.SPMV_ACC_SEGMENT)
                    t1.record()
                    torch.cuda.synchronize()
                    sweep.append({"tau": tau, "ms": round(t0.elapsed_time(t1) / 5, 4),
                                  "max_accumulation_err": rel_err(y.double().cpu().numpy(), y_ref, s_ref)})
                full = sweep[0]["max_accumulation_err"]
                ok = [e for e in sweep if e["max_accumulation_err"] <= 1.5 * full]
                entry["tau_sweep"] = {"product": "row-split, FP32 values and vectors, SPMV_ACC_SEGMENT",
                                      "rule": "largest tau whose error stays within 1.5x of compensating every row",
                                      "chosen_tau": max(e["tau"] for e in ok), "points": sweep}
            sp.spmv_destroy(h)
        out.append(entry)
        del rp, co, vo
    return out


TAUS = (0, 2, 4, 8, 16, 32, 2048, 1 << 40)


# ------------------------------------------------------------------ main

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=RMAT["scale"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle", action="store_true", help="skip the oracle's errors and CPU baselines")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-precision", action="store_true")
    ap.add_argument("--no-iterative", action="store_true")
    ap.add_argument("--no-blocking", action="store_true", help="skip the Merge Blocking leg")
    ap.add_argument("--batched-small", action="store_true", help="64 matrices, scales 10-18")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    import numpy as np
    import synth

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import torch.distributed as dist
    import paper_2502_19284_gb300 as sp

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)

    # each rank runs its own instance of the workload (independent problems: weak scaling)
    scale = args.scale
    m = n = 1 << scale
    rows, cols = synth.rmat(scale, RMAT["edge_factor"], seed=rank, abcd=RMAT["abcd"])
    vals = synth.values(rows, cols, seed=rank)
    x = synth.vector(n, seed=rank + 1)
    nnz_in = int(rows.size)
    r_d = torch.from_numpy(rows).to(dev)
    c_d = torch.from_numpy(cols).to(dev)
    v_d = torch.from_numpy(vals).to(dev)
    x_d = torch.from_numpy(x).to(dev)
    ys = {p: torch.empty(m, dtype=torch.float64, device=dev) for p in PRODUCTS}
    flush = torch.empty(FLUSH_BYTES // 4, dtype=torch.int32, device=dev)

    ev = lambda: torch.cuda.Event(enable_timing=True)
    stages = ["ingest", "coo_to_csr", "spmv_rowsplit", "merge_partition", "spmv_merge", "spmv_merge_f64",
              "csr_to_hb", "spmv_hb"]
    hb_opts = dict(log2_beta=14)

    def step(rec, src=None, host_x=None, host_y=None):
        # src: host (pinned) triplets for the end-to-end variant of the whole step
        e = {st: (ev(), ev()) for st in stages}

        def run(st, fn):
            e[st][0].record()
            fn()
            e[st][1].record()

        def product(st, algo_acc):
            flush.fill_(1)                          # L2 flush, outside the product's events
            if host_x is not None:
                x_d.copy_(host_x, non_blocking=True)
            run(st, lambda: sp.spmv_mul(h, x_d, ys[st], accum=algo_acc))
            if host_y is not None:
                host_y[st].copy_(ys[st], non_blocking=True)

        box = {}
        run("ingest", lambda: box.setdefault("h", sp.spmv_create_coo(m, n, r_d, c_d, v_d) if src is None
                                              else sp.spmv_create_coo(m, n, *src)))
        h = box["h"]
        run("coo_to_csr", lambda: sp.spmv_convert(h, "rowsplit"))
        product("spmv_rowsplit", sp.SPMV_ACC_DEFAULT)
        run("merge_partition", lambda: sp.spmv_convert(h, "merge"))
        product("spmv_merge", sp.SPMV_ACC_DEFAULT)
        product("spmv_merge_f64", sp.SPMV_ACC_F64)
        run("csr_to_hb", lambda: sp.spmv_convert(h, "hb", **hb_opts))
        product("spmv_hb", sp.SPMV_ACC_DEFAULT)
        info = sp.spmv_info(h)
        sp.spmv_destroy(h)
        rec.append((e, info))

    def timed(K, W, trace=False, **kw):
        for _ in range(W):
            step([], **kw)
        torch.cuda.synchronize()
        if trace:
            sp.spmv_trace_enable(True)   # clears the table; synchronises the device
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        recs = []
        t0, t1 = ev(), ev()
        w0 = time.perf_counter()
        t0.record()
        for _ in range(K):
            step(recs, **kw)
        t1.record()
        torch.cuda.synchronize()
        wall = time.perf_counter() - w0
        if world > 1:
            dist.barrier()
        return t0.elapsed_time(t1), wall, recs

    # ---- device-resident timed region (with the library's kernel trace on)
    with ClockSampler(local) as clk:
        total_ms, wall_s, recs = timed(args.steps, args.warmup, trace=True)
        trace = sp.spmv_trace_read()
        sp.spmv_trace_enable(False)
    info = recs[-1][1]
    nnz, nblk = info["nnz"], info["nblk"]
    rb = row_bytes(m, n, nnz, nblk)
    step_bytes = sum(rb.values())
    ms_step = max_over_ranks(total_ms / args.steps, world, dist, dev)
    per = {st: statistics.median(e[st][0].elapsed_time(e[st][1]) for e, _ in recs) for st in stages}
    per = {st: max_over_ranks(v, world, dist, dev) for st, v in per.items()}
    sb = spmv_bytes(m, n, nnz)
    rows_out = {}
    for st in stages:
        d = {"ms": round(per[st], 4), "gbs": round(rb[st] / (per[st] * 1e-3) / 1e9, 1) if rb[st] else None}
        if st in PRODUCTS:
            d["gflops"] = round(2 * nnz / (per[st] * 1e-3) / 1e9, 1)
            d["what"] = PRODUCT_DESC[st]
        rows_out[st] = d
    fp64 = ["spmv_rowsplit", "spmv_merge", "spmv_merge_f64", "spmv_hb"]
    best = max(fp64, key=lambda st: rb[st] / per[st])      # highest compulsory-byte rate
    value = job_value(rb[best], per[best], world)
    best_csr = max(["spmv_rowsplit", "spmv_merge", "spmv_merge_f64"], key=lambda st: rb[st] / per[st])

    # ---- roofline of each product's main kernel (device time from the library's trace)
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "of measured" if peak else "of fallback"
    peak = peak or FALLBACK_HBM_GBS
    traffic_db = {}
    try:
        traffic_db = json.load(open(os.path.join(ROOT, "profiles", "ncu_traffic.json")))
    except (OSError, ValueError):
        pass

    def roofline_for(kname):
        if kname not in trace:
            return None
        cnt, kms = trace[kname]
        kb = kernel_bytes(kname, m, n, nnz, nblk)
        if kb is None or cnt == 0:
            return None
        per_launch = kb * args.steps / cnt          # algorithmic bytes of an average launch
        dur = kms / cnt                             # its average duration (CUDA events, ms)
        ach = per_launch / (dur * 1e-3) / 1e9
        traffic = None
        t = traffic_db.get(kname)
        units = kernel_units(kname, m, n, nnz)
        if t and units and t.get("source_sha") == source_sha(t.get("source"), t.get("from"), t.get("to")):
            traffic = int(t["bytes_per_unit"] * units * args.steps / cnt)   # ncu DRAM bytes, scaled per launch
        return {"kernel": kname, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_note": peak_src, "traffic": traffic,
                "algorithmic_bytes_per_launch": int(per_launch), "launches": cnt, "avg_launch_ms": round(dur, 5)}

    roof = roofline_for(PRODUCT_KERNEL[best])
    roof_products = {st: roofline_for(PRODUCT_KERNEL[st]) for st in PRODUCTS}
    for st in PRODUCTS:
        rows_out[st]["frac_of_peak"] = round(rb[st] / (per[st] * 1e-3) / 1e9 / peak, 4)
    dominant = max(trace, key=lambda k: trace[k][1])
    roof_dom = roofline_for(dominant)
    launches = sum(c for c, _ in trace.values())
    tot_ms = sum(u[1] for u in trace.values())
    shares = {k: round(v[1] / tot_ms, 4) for k, v in sorted(trace.items(), key=lambda kv: -kv[1][1])}

    # ---- break-even count of the blocked format against the faster CRS product
    from paper_2502_19284_gb300 import breakeven
    t_csr_best = min(per["spmv_rowsplit"], per["spmv_merge"], per["spmv_merge_f64"])
    ns_ = breakeven.n_star_times(per["csr_to_hb"], 0.0, t_csr_best, per["spmv_hb"])
    break_even = {"n_star_gpu": None if ns_ is None else round(ns_, 1),
                  "meaning": "SpMVs after which CSR->HB conversion pays back against the faster CRS product "
                             "(None: the blocked product is not faster)"}

    # ---- end to end through the public API with host buffers: the converted matrix stays
    # resident; every iteration copies x in from pinned host memory, multiplies with the
    # product the value names and reads y back
    e2e = None
    e2e_step = None
    if not args.no_e2e:
        hx = torch.from_numpy(x).pin_memory()
        hy = torch.empty(m, dtype=torch.float64).pin_memory()
        h = sp.spmv_create_coo(m, n, r_d, c_d, v_d)
        fmt = {"spmv_rowsplit": "rowsplit", "spmv_hb": "hb"}.get(best, "merge")
        sp.spmv_convert(h, fmt, **(hb_opts if fmt == "hb" else {}))
        acc = sp.SPMV_ACC_F64 if best == "spmv_merge_f64" else sp.SPMV_ACC_DEFAULT
        yd = ys[best]

        def once():
            x_d.copy_(hx, non_blocking=True)
            sp.spmv_mul(h, x_d, yd, accum=acc)
            hy.copy_(yd, non_blocking=True)
        for _ in range(3):
            once()
        torch.cuda.synchronize()
        K2 = max(10, 5 * args.steps)
        t0, t1 = ev(), ev()
        t0.record()
        for _ in range(K2):
            once()
        t1.record()
        torch.cuda.synchronize()
        ms_serial = max_over_ranks(t0.elapsed_time(t1) / K2, world, dist, dev)
        # the same steps with consecutive steps overlapped: x in, the product and y out on three
        # streams with two device buffers each; events order every copy against the product that
        # uses its buffer, and the products run one after another (the handle's scratch is shared)
        s_in, s_cp, s_out = torch.cuda.Stream(), torch.cuda.Stream(), torch.cuda.Stream()
        xb = [torch.empty(n, dtype=torch.float64, device=dev) for _ in range(2)]
        yb = [torch.empty(m, dtype=torch.float64, device=dev) for _ in range(2)]
        hyb = [torch.empty(m, dtype=torch.float64).pin_memory() for _ in range(2)]
        e_in = [torch.cuda.Event() for _ in range(2)]
        e_cp = [torch.cuda.Event() for _ in range(2)]
        e_out = [torch.cuda.Event() for _ in range(2)]
        for e in e_cp + e_out:
            e.record(torch.cuda.current_stream())

        def piped(i):
            b = i & 1
            s_in.wait_event(e_cp[b])                 # the product two steps back has read xb[b]
            with torch.cuda.stream(s_in):
                xb[b].copy_(hx, non_blocking=True)
            e_in[b].record(s_in)
            s_cp.wait_event(e_in[b])
            s_cp.wait_event(e_out[b])                # y of two steps back has left yb[b]
            sp.spmv_mul(h, xb[b], yb[b], accum=acc, stream=s_cp)
            e_cp[b].record(s_cp)
            s_out.wait_event(e_cp[b])
            with torch.cuda.stream(s_out):
                hyb[b].copy_(yb[b], non_blocking=True)
            e_out[b].record(s_out)
        for i in range(4):
            piped(i)
        torch.cuda.synchronize()
        t0.record()
        for st_ in (s_in, s_cp, s_out):
            st_.wait_stream(torch.cuda.current_stream())   # no step starts before t0
        for i in range(K2):
            piped(i)
        for st_ in (s_in, s_cp, s_out):
            torch.cuda.current_stream().wait_stream(st_)
        t1.record()
        torch.cuda.synchronize()
        ms_e = max_over_ranks(t0.elapsed_time(t1) / K2, world, dist, dev)
        piped_diff = float(np.max(np.abs(hyb[(K2 - 1) & 1].numpy() - hy.numpy())))   # against a serial step
        sp.spmv_destroy(h)
        e2e = {"value": round(job_value(rb[best], ms_e, world), 2), "unit": "GB/s",
               "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": m * 8, "ms_per_step": round(ms_e, 4),
               "what": (f"{best}: every step x host->device from pinned memory, spmv_mul, y device->host to pinned "
                        "memory, matrix resident; consecutive steps overlapped on three streams (copies in and "
                        "out beside the previous and next products)"),
               "max_abs_diff_vs_serial": piped_diff,
               "serial": {"value": round(job_value(rb[best], ms_serial, world), 2), "ms_per_step": round(ms_serial, 4),
                          "what": "the same steps one after another on one stream"}}
        # the whole step from host triplets (matrix ingest over the host link included)
        hr = torch.from_numpy(rows).pin_memory()
        hc = torch.from_numpy(cols).pin_memory()
        hv = torch.from_numpy(vals).pin_memory()
        hys = {st: torch.empty(m, dtype=torch.float64).pin_memory() for st in PRODUCTS}
        K3 = max(2, args.steps // 4)
        tot3, _, _ = timed(K3, 1, src=(hr, hc, hv), host_x=hx, host_y=hys)
        ms3 = max_over_ranks(tot3 / K3, world, dist, dev)
        e2e_step = {"ms_per_step": round(ms3, 3), "step_gbs": round(job_value(step_bytes, ms3, world), 2),
                    "h2d_bytes_per_step": nnz_in * 16 + 4 * n * 8, "d2h_bytes_per_step": 4 * m * 8}
        del hr, hc, hv, hys

    # ---- Merge Blocking (Section 4.3) on the same workload, outside the timed step
    blocking, ys_mb = (None, {}) if args.no_blocking else blocking_leg(sp, torch, dev, m, n, r_d, c_d, v_d, x_d,
                                                                       flush, traffic_db)
    if blocking:
        for fmt in ("mergeb", "mergebh"):
            kg = blocking[fmt]["kernel_gbs"]
            blocking[fmt]["kernel_frac_of_peak"] = None if kg is None else round(kg / peak, 4)
            blocking[fmt]["frac_of_peak"] = round(blocking[fmt]["gbs"] / peak, 4)

    # ---- errors of every product against the oracle, CPU baselines (rank 0)
    errors = None
    cpu = None
    if rank == 0 and not args.no_oracle:
        ref = OracleCSR(m, n, rows, cols, vals, x)
        errors = {st: rel_err(ys[st].cpu().numpy(), ref.y, ref.scale) for st in PRODUCTS}
        for st in PRODUCTS:
            rows_out[st]["max_err"] = errors[st]
        for fmt, y in ys_mb.items():
            errors[fmt] = rel_err(y.cpu().numpy(), ref.y, ref.scale)
            blocking[fmt]["max_err"] = errors[fmt]
        if world == 1 and not args.no_cpu_baseline:
            cpu = cpu_baselines(ref)
        del ref

    # ---- extension legs (outside the timed region)
    serving = None if args.no_serving else serving_leg(sp, torch, dev, synth, np)
    batched = None if args.no_batched else batched_leg(sp, torch, dev, synth, np,
                                                         BATCH_SMALL if args.batched_small else BATCH)
    precision = None if args.no_precision else precision_leg(sp, torch, dev, synth, np)
    iterative = None if args.no_iterative else iterative_leg(sp, torch, dev, synth, np)

    if world > 1:
        dist.destroy_process_group()
    if rank != 0:
        return 0
    out = {
        "metric": METRIC,
        "value": round(value, 2),
        "unit": "GB/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms_step, 4),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_desc(scale), "m": m, "n": n, "nnz": nnz, "triplets": nnz_in, "nblk": nblk,
                   "log2_beta": info["log2_beta"],
                   "value": (f"compulsory bytes of {best} ({rb[best]} B: {PRODUCT_DESC[best]}) / its device time "
                             "inside the step, median of the timed steps"),
                   "value_from": best, "value_csr": round(job_value(rb[best_csr], per[best_csr], world), 2),
                   "value_csr_from": best_csr,
                   "step": "ingest -> COO->CSR + bins -> row-split SpMV -> merge partition -> merge SpMV (double-float) "
                           "-> merge SpMV (native FP64) -> CSR->HB (beta 2^14) -> HB SpMV -> destroy",
                   "step_bytes": step_bytes, "step_gbs": round(job_value(step_bytes, ms_step, world), 2),
                   "l2": "flushed (256 MB write) before every product; triplets 1 GB per step",
                   "parallelism": f"replicas x{world}"},
        "rows": rows_out,
        "clocks": clk.summary(),
        "e2e": e2e,
        "e2e_step": e2e_step,
        "gpu_launches": launches,
        "roofline": roof,
        "roofline_products": roof_products,
        "roofline_step_dominant": roof_dom,
        "kernel_shares": shares,
        "break_even": break_even,
        "errors_vs_oracle": errors,
        "merge_blocking": blocking,
        "serving": serving,
        "batched": batched,
        "precision": precision,
        "iterative": iterative,
        "cpu_baseline": cpu,
        "wall_s_timed": round(wall_s, 3),
    }
    print(json.dumps(out), flush=True)
    return 0


def source_sha(rel, start=None, end=None):
    """Hash of a kernel's source: the file, or the text between two marker lines of it."""
    if not rel:
        return None
    try:
        text = open(os.path.join(ROOT, rel), "rb").read()
    except OSError:
        return None
    if start:
        i = text.find(start.encode())
        j = text.find(end.encode(), i + 1) if end and i >= 0 else -1
        if i < 0 or j < 0:
            return None
        text = text[i:j]
    return hashlib.sha256(text).hexdigest()[:16]


def run_reference(args, rank, world):
    """Reference arm: the oracle, as it stands, on one host core: each step is Algorithm 1 on
    the full matrix of the workload (the CRS arrays come from the oracle's own COO->CSR,
    built once before the warm-up), K timed steps, rank 0 only."""
    if rank != 0:
        return 0
    import synth
    scale = args.scale
    m = n = 1 << scale
    rows, cols = synth.rmat(scale, RMAT["edge_factor"], seed=0, abcd=RMAT["abcd"])
    vals = synth.values(rows, cols, seed=0)
    x = synth.vector(n, seed=1)
    ref = OracleCSR(m, n, rows, cols, vals, x)
    import oracle
    for _ in range(args.warmup):
        oracle.csr_spmv(ref.rp, ref.co, ref.vo, x)
    times = []
    for _ in range(args.steps):
        t = time.perf_counter()
        oracle.csr_spmv(ref.rp, ref.co, ref.vo, x)
        times.append(time.perf_counter() - t)
    b = spmv_bytes(m, n, ref.nnz)
    ms = 1e3 * statistics.median(times)
    value = b / (ms * 1e-3) / 1e9
    desc = (f"the full R-MAT scale-{scale} matrix ({ref.nnz} nonzeros), Algorithm 1 on one core per step "
            f"(median {ms:.1f} ms); the oracle's COO->CSR before the warm-up took {ref.coo_to_csr_s:.2f} s")
    out = {
        "impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "GB/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(scale), "m": m, "n": n, "nnz": ref.nnz,
                   "value": "compulsory bytes of one FP64 CSR product / the oracle's time for it"},
        "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
