"""Pins of the CPU oracle against things other than itself (runs without a GPU).

Each test checks one oracle function against values printed in the paper (golden
fixtures under tests/golden/, each citing its figure or table), against closed forms,
against brute force on tiny inputs, or against invariants -- chosen so that a
plausible mistake (a dropped term, a wrong sign or index, a transposed operand)
fails at least one of them.  The `test_planted_*` cases show that the pins do bite.
"""
import math
import os
import re
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from conftest import golden_path


# ------------------------------------------------------------------ figure decoding

def _read_curves(name):
    """Parse a figure fixture into {order: [(row, col) cell per curve position]}."""
    curves = {}
    order = None
    for line in open(golden_path(name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("order"):
            order = int(line.split()[1])
            continue
        pts = [(float(a), float(b)) for a, b in re.findall(r"\(([-0-9.]+),([-0-9.]+)\)", line)]
        S = 1 << order
        w = 4.0 / S
        cells = []
        for x, y in pts:
            col = x / w - 0.5
            row = (4.0 - y) / w - 0.5
            assert abs(col - round(col)) < 1e-9 and abs(row - round(row)) < 1e-9
            cells.append((int(round(row)), int(round(col))))
        curves[order] = cells
    return curves


def _expand_axis_path(vertices):
    """Cells visited by a path of axis-aligned straight segments through cell centres."""
    out = [vertices[0]]
    for (r0, c0), (r1, c1) in zip(vertices, vertices[1:]):
        assert r0 == r1 or c0 == c1, "Hilbert figure segments are axis-aligned"
        dr = (r1 > r0) - (r1 < r0)
        dc = (c1 > c0) - (c1 < c0)
        r, c = r0, c0
        while (r, c) != (r1, c1):
            r, c = r + dr, c + dc
            out.append((r, c))
    return out


def _figure_table(cells, order):
    S = 1 << order
    t = -np.ones((S, S), np.int64)
    for i, (r, c) in enumerate(cells):
        t[r, c] = i
    assert (t >= 0).all() and len(cells) == S * S
    return t


def hilbert_figure_tables():
    return {k: _figure_table(_expand_axis_path(v), k) for k, v in _read_curves("hilbert_figure.txt").items()}


def zmorton_figure_tables():
    return {k: _figure_table(v, k) for k, v in _read_curves("zmorton_figure.txt").items()}


# ------------------------------------------------------------------ Hilbert curve

def test_hilbert_matches_paper_figure(orc):
    tabs = hilbert_figure_tables()
    assert set(tabs) == {1, 2, 3}
    for K, t in tabs.items():
        np.testing.assert_array_equal(oracle.hilbert_table(K, orc), t, err_msg=f"order {K}")


@pytest.mark.parametrize("K", [1, 2, 3, 4, 5, 6, 7])
def test_hilbert_properties(orc, K):
    t = oracle.hilbert_table(K, orc)
    S = 1 << K
    # bijection onto 0 .. 4^K - 1
    assert sorted(t.ravel().tolist()) == list(range(S * S))
    pos = np.empty((S * S, 2), np.int64)
    for r in range(S):
        for c in range(S):
            pos[t[r, c]] = (r, c)
    # consecutive cells are 4-neighbours: exactly one index changes, by one (Section 4.1)
    steps = np.abs(np.diff(pos, axis=0)).sum(axis=1)
    assert (steps == 1).all()
    # enters at the top-left cell, leaves at the top-right cell (figure)
    assert tuple(pos[0]) == (0, 0) and tuple(pos[-1]) == (0, S - 1)
    # every aligned 2^b square is one contiguous range of the curve (recursive definition)
    for b in range(1, K):
        B = 1 << b
        for r0 in range(0, S, B):
            for c0 in range(0, S, B):
                blk = t[r0:r0 + B, c0:c0 + B].ravel()
                assert blk.max() - blk.min() == B * B - 1
                assert blk.min() % (B * B) == 0


def test_hilbert_large_grid_block_property(orc):
    """At K = 22 (the scale-22 grid), the top 2(K-b) bits of h give the block, and the
    block order is the order-(K-b) curve on block coordinates."""
    rng = np.random.default_rng(3)
    K, b = 22, 14
    for _ in range(2000):
        r, c = (int(v) for v in rng.integers(0, 1 << K, size=2))
        h = oracle.hilbert_index(K, r, c, orc)
        assert 0 <= h < 1 << (2 * K)
        assert h >> (2 * b) == oracle.hilbert_index(K - b, r >> b, c >> b, orc)


def test_zmorton_matches_paper_figure(orc):
    tabs = zmorton_figure_tables()
    for K, t in tabs.items():
        np.testing.assert_array_equal(oracle.zmorton_table(K, orc), t, err_msg=f"order {K}")


# ------------------------------------------------------------------ block size rule

def test_block_size_rule_closed_form(orc):
    # Eq. 2 upper bound 3 + ceil(log2 sqrt n): n = 2^22 -> 14, n = 2^16 -> 11, n = 2^23 -> 15
    # (then limited by the on-chip slice: 2^15 doubles = 256 KiB > 200 KiB -> 14).
    assert oracle.log2_beta(1 << 22, 8, 1 << 30, orc) == 14
    assert oracle.log2_beta(1 << 16, 8, 1 << 30, orc) == 11
    assert oracle.log2_beta(1 << 23, 8, 1 << 30, orc) == 15
    assert oracle.log2_beta(1 << 23, 8, 200 * 1024, orc) == 14
    # 16-bit packing limit: n = 2^30 -> 3 + 15 = 18 -> capped at 16
    assert oracle.log2_beta(1 << 30, 8, 1 << 40, orc) == 16
    # not a power of two: n = 5e6 -> ceil(log2 n) = 23 -> ceil(23/2) = 12 -> 15
    assert oracle.log2_beta(5_000_000, 4, 1 << 30, orc) == 15
    for n in [2, 3, 100, 1000, 12345, 1 << 20]:
        b = oracle.log2_beta(n, 8, 1 << 40, orc)
        lower = math.ceil(math.log2(math.sqrt(n)) - 1e-12)
        assert max(4, lower) <= b <= 3 + lower + 1e-9 or b == 4


# ------------------------------------------------------------------ merge path

def _read_merge_fixture():
    d = {}
    for line in open(golden_path("merge_path_figure.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, _, v = line.partition(" ")
        d[k] = v.strip()
    A = [int(v) for v in d["A"].split()]
    B = [int(v) for v in d["B"].split()]
    nodes = [(int(a), int(b)) for a, b in re.findall(r"\((\d+),(\d+)\)", d["nodes"])]
    return A, B, int(d["threads"]), [(x, 4 - y) for x, y in nodes], d["consumed"].split()


def test_merge_path_matches_paper_figure(orc):
    A, B, threads, nodes, consumed = _read_merge_fixture()
    # every node of the drawn path is the walk's state after that many steps
    for d, node in enumerate(nodes):
        assert oracle.merge_path_walk(d, A, B, orc) == node
    # three threads, four steps each: split points are nodes 0, 4, 8, 12
    total = len(A) + len(B)
    per = total // threads
    splits = [oracle.merge_path_walk(t * per, A, B, orc) for t in range(threads + 1)]
    assert splits == [(0, 0), (3, 1), (5, 3), (8, 4)]
    # the consumed sequence (ties go to list A)
    seq = []
    for (a0, b0), (a1, b1) in zip(nodes, nodes[1:]):
        seq.append(f"A{A[a0]}" if a1 > a0 else f"B{B[b0]}")
    assert seq == consumed


def _random_csr(m, n, nnz, seed, integer=False):
    r, c = synth.random_coo(m, n, nnz, seed)
    v = synth.values(r, c, seed, integer=integer)
    rp, co, vo = oracle.coo_to_csr(m, n, r, c, v)
    return rp, co, vo


@pytest.mark.parametrize("seed", range(6))
def test_merge_path_search_equals_walk(orc, seed):
    """Bisection split == the plain walk with A = row ends, B = 0..nnz-1, every diagonal."""
    rng = np.random.default_rng(seed)
    m = int(rng.integers(1, 40))
    n = int(rng.integers(1, 40))
    rp, co, _ = _random_csr(m, n, int(rng.integers(0, 3 * m)), seed)
    nnz = int(rp[-1])
    A = rp[1:].astype(np.int64)
    B = np.arange(nnz, dtype=np.int64)
    for d in range(m + nnz + 1):
        assert oracle.merge_path_search(d, rp, orc) == oracle.merge_path_walk(d, A, B, orc)


# ------------------------------------------------------------------ COO -> CRS

def _brute_csr(m, rows, cols, vals):
    ent = {}
    for i, (r, c) in enumerate(zip(rows.tolist(), cols.tolist())):
        ent.setdefault((r, c), []).append(vals[i])
    keys = sorted(ent)
    rp = np.zeros(m + 1, np.int64)
    for r, _ in keys:
        rp[r + 1] += 1
    rp = np.cumsum(rp)
    co = np.array([c for _, c in keys], np.int64)
    vo = []
    for k in keys:
        s = 0.0
        for v in ent[k]:          # duplicates summed in input order
            s = s + v
        vo.append(s)
    return rp, co, np.array(vo)


@pytest.mark.parametrize("seed", range(8))
def test_coo_to_csr_brute_force(orc, seed):
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(1, 30)), int(rng.integers(1, 30))
    rows, cols = synth.random_coo(m, n, int(rng.integers(0, 120)), seed, dup_frac=0.3 if seed % 2 else 0.0)
    vals = rng.standard_normal(rows.shape[0])
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    brp, bco, bvo = _brute_csr(m, rows, cols, vals)
    np.testing.assert_array_equal(rp, brp)
    np.testing.assert_array_equal(co, bco)
    np.testing.assert_array_equal(vo, bvo)      # same addition order: bit-exact
    # invariants
    assert rp[0] == 0 and rp[-1] == co.shape[0] and (np.diff(rp) >= 0).all()
    for i in range(m):
        assert (np.diff(co[rp[i]:rp[i + 1]]) > 0).all()


def test_coo_to_csr_errors(orc):
    with pytest.raises(oracle.OracleError) as e:
        oracle.coo_to_csr(3, 3, [0, 3], [0, 0], [1.0, 2.0], 0, orc)
    assert e.value.code == oracle.ERR_INDEX_RANGE
    with pytest.raises(oracle.OracleError) as e:
        oracle.coo_to_csr(3, 3, [1, 1], [2, 2], [1.0, 2.0], 1, orc)
    assert e.value.code == oracle.ERR_DUPLICATE
    rp, co, vo = oracle.coo_to_csr(4, 5, [], [], [], 0, orc)
    assert rp.tolist() == [0] * 5 and co.size == 0


# ------------------------------------------------------------------ Algorithm 1

def _dense(m, n, rp, co, vo):
    D = np.zeros((m, n))
    for i in range(m):
        for k in range(rp[i], rp[i + 1]):
            D[i, co[k]] += vo[k] if vo is not None else 1.0
    return D


@pytest.mark.parametrize("seed", range(10))
def test_csr_spmv_integer_brute_force(orc, seed):
    """Integer values and x: every partial sum is exact, so y equals the dense product exactly."""
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 64)), int(rng.integers(1, 64))
    rp, co, vo = _random_csr(m, n, int(rng.integers(0, 4 * m + 1)), seed, integer=True)
    x = synth.vector(n, seed + 1, integer=True)
    D = _dense(m, n, rp, co, vo).astype(np.int64)
    yref = D @ x.astype(np.int64)
    np.testing.assert_array_equal(oracle.csr_spmv(rp, co, vo, x, orc), yref.astype(np.float64))
    # pattern matrix: values implicitly 1
    P = (D != 0).astype(np.int64) if vo is not None else D
    Dp = _dense(m, n, rp, co, None).astype(np.int64)
    np.testing.assert_array_equal(oracle.csr_spmv(rp, co, None, x, orc), (Dp @ x.astype(np.int64)).astype(float))
    del P


@pytest.mark.parametrize("seed", range(6))
def test_csr_spmv_float_exact_sum(orc, seed):
    """Floating values: Algorithm 1 is the left-to-right sum of correctly rounded
    products; compare with exact rational arithmetic of that same order."""
    rng = np.random.default_rng(50 + seed)
    m, n = int(rng.integers(1, 20)), int(rng.integers(1, 20))
    rp, co, vo = _random_csr(m, n, int(rng.integers(0, 5 * m + 1)), seed)
    x = synth.vector(n, seed + 1)
    y = oracle.csr_spmv(rp, co, vo, x, orc)
    for i in range(m):
        s = 0.0
        exact = Fraction(0)
        for k in range(rp[i], rp[i + 1]):
            p = float(vo[k]) * float(x[co[k]])       # one rounding per product
            s = s + p                                 # one rounding per addition
            exact += Fraction(vo[k]) * Fraction(x[co[k]])
        assert y[i] == s
        L = rp[i + 1] - rp[i]
        bound = L * 2.0 ** -53 / (1 - L * 2.0 ** -53) * sum(abs(vo[k] * x[co[k]]) for k in range(rp[i], rp[i + 1]))
        assert abs(Fraction(y[i]) - exact) <= Fraction(bound) * (1 + 1e-12) + Fraction(1, 10 ** 300)


def test_csr_spmv_equals_triplet_eq1(orc):
    rng = np.random.default_rng(9)
    m, n = 50, 40
    rows, cols = synth.random_coo(m, n, 300, 9)
    vals = synth.values(rows, cols, 9, integer=True)
    x = synth.vector(n, 10, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    np.testing.assert_array_equal(oracle.csr_spmv(rp, co, vo, x, orc), oracle.coo_spmv(m, rows, cols, vals, x, orc))
    del rng


def test_invariants_row_sums_and_adjoint(orc):
    rows, cols = synth.rmat(10, 8, seed=4)
    m = n = 1 << 10
    vals = synth.values(rows, cols, 4)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    # A 1 = row sums of data (exact for integer data; here compare to fsum within rounding)
    y1 = oracle.csr_spmv(rp, co, vo, np.ones(n), orc)
    for i in range(0, m, 7):
        ref = math.fsum(vo[rp[i]:rp[i + 1]])
        assert abs(y1[i] - ref) <= 1e-13 * max(1.0, np.abs(vo[rp[i]:rp[i + 1]]).sum())
    # x^T (A y) = (A^T x)^T y
    x = synth.vector(m, 11)
    yv = synth.vector(n, 12)
    trp, tco, tvo = oracle.csr_transpose(m, n, rp, co, vo, orc)
    lhs = math.fsum(x * oracle.csr_spmv(rp, co, vo, yv, orc))
    rhs = math.fsum(oracle.csr_spmv(trp, tco, tvo, x, orc) * yv)
    scale = math.fsum(np.abs(x) * oracle.csr_absmul(rp, co, vo, np.abs(yv), orc))
    assert abs(lhs - rhs) <= 1e-12 * scale


def test_transpose_brute_force(orc):
    m, n = 13, 17
    rp, co, vo = _random_csr(m, n, 60, 5)
    trp, tco, tvo = oracle.csr_transpose(m, n, rp, co, vo, orc)
    np.testing.assert_array_equal(_dense(n, m, trp, tco, tvo), _dense(m, n, rp, co, vo).T)


def test_neumaier_against_fsum(orc):
    # one row whose terms cancel: plain summation loses everything, compensated keeps it
    terms = np.array([1e16, 1.0, -1e16, 3.0, 1e-3, -2.0])
    rp = np.array([0, terms.size], np.int32)
    co = np.arange(terms.size, dtype=np.int32)
    x = np.ones(terms.size)
    y = oracle.csr_spmv_neumaier(rp, co, terms, x, orc)
    assert y[0] == math.fsum(terms)
    rng = np.random.default_rng(2)
    for _ in range(20):
        t = rng.standard_normal(200) * 10.0 ** rng.integers(-5, 5, 200)
        y = oracle.csr_spmv_neumaier(np.array([0, 200], np.int32), np.arange(200, dtype=np.int32), t, np.ones(200), orc)
        assert abs(y[0] - math.fsum(t)) <= 2 * 2.0 ** -53 * abs(math.fsum(t)) + 1e-300


# ------------------------------------------------------------------ CRS -> blocked

def _hb_to_triplets(hb):
    out = []
    b = hb["log2beta"]
    for k in range(hb["nblk"]):
        r0, c0 = int(hb["blk_row"][k]) << b, int(hb["blk_col"][k]) << b
        for t in range(hb["blk_ptr"][k], hb["blk_ptr"][k + 1]):
            out.append((r0 + (int(hb["idx"][t]) >> 16), c0 + (int(hb["idx"][t]) & 0xFFFF),
                        hb["val"][t] if hb["val"] is not None else 1.0))
    return out


@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_csr_to_hb_structure_and_round_trip(orc, seed, inner):
    rng = np.random.default_rng(seed)
    m, n = int(rng.integers(1, 70)), int(rng.integers(1, 70))
    rp, co, vo = _random_csr(m, n, int(rng.integers(0, 6 * m + 1)), seed)
    K = oracle.grid_order(m, n, orc)
    for lb in [1, 2, 3]:
        hb = oracle.csr_to_hb(m, n, rp, co, vo, lb, inner, orc)
        b = hb["log2beta"]
        trip = _hb_to_triplets(hb)
        # round trip back to CRS is bit-exact
        ref = sorted((i, int(co[k]), vo[k]) for i in range(m) for k in range(rp[i], rp[i + 1]))
        assert sorted(trip) == ref
        # blocks are contiguous runs; block coordinates consistent; Hilbert block order
        prev = -1
        for k in range(hb["nblk"]):
            assert hb["blk_ptr"][k] < hb["blk_ptr"][k + 1]
            hblk = oracle.hilbert_index(K - b, int(hb["blk_row"][k]), int(hb["blk_col"][k]), orc)
            assert hblk > prev
            prev = hblk
        # entry order inside blocks: Hilbert (inner 0) or row-wise (inner 1)
        for k in range(hb["nblk"]):
            ent = trip[hb["blk_ptr"][k]:hb["blk_ptr"][k + 1]]
            if inner == 0:
                keys = [oracle.hilbert_index(K, r, c, orc) for r, c, _ in ent]
            else:
                keys = [(r, c) for r, c, _ in ent]
            assert keys == sorted(keys) and len(set(keys)) == len(keys)


@pytest.mark.parametrize("seed", range(4))
def test_hb_spmv_integer_equals_alg1(orc, seed):
    rows, cols = synth.rmat(9, 8, seed=seed)
    m = n = 1 << 9
    vals = synth.values(rows, cols, seed, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    x = synth.vector(n, seed + 1, integer=True)
    hb = oracle.csr_to_hb(m, n, rp, co, vo, 5, 0, orc)
    np.testing.assert_array_equal(oracle.hb_spmv(m, hb, x, orc), oracle.csr_spmv(rp, co, vo, x, orc))


# ------------------------------------------------------------------ merge-based SpMV

@pytest.mark.parametrize("parts", [1, 2, 3, 7, 64, 1000])
def test_merge_spmv(orc, parts):
    rows, cols = synth.rmat(9, 8, seed=1)
    m = n = 1 << 9
    vals = synth.values(rows, cols, 1, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    x = synth.vector(n, 2, integer=True)
    y, cr, cv = oracle.merge_spmv(rp, co, vo, x, parts, orc)
    np.testing.assert_array_equal(y, oracle.csr_spmv(rp, co, vo, x, orc))
    # float data: same result up to summation order
    vf = synth.values(rows, cols, 1)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vf, 0, orc)
    xf = synth.vector(n, 2)
    y, _, _ = oracle.merge_spmv(rp, co, vo, xf, parts, orc)
    ref = oracle.csr_spmv(rp, co, vo, xf, orc)
    scale = oracle.csr_absmul(rp, co, vo, xf, orc)
    assert (np.abs(y - ref) <= 1e-13 * scale).all()


# ------------------------------------------------------------------ precision

def _bf16_grid():
    bits = np.arange(0, 0x7F80, dtype=np.uint32)          # all finite non-negative bfloat16
    return (bits << 16).view(np.float32).astype(np.float64)


def test_round_bf16_nearest_even_brute_force(orc):
    grid = _bf16_grid()
    rng = np.random.default_rng(0)
    vals = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-40, 38, 3000),
                           (grid[1:200] + grid[:199]) / 2,          # exact ties
                           grid[rng.integers(1, grid.size - 1, 500)]])
    for v in vals:
        a = abs(float(v))
        if a > grid[-1]:
            continue
        i = np.searchsorted(grid, a)
        cand = [grid[j] for j in (i - 1, i) if 0 <= j < grid.size]
        best = min(cand, key=lambda g: (abs(Fraction(g) - Fraction(a)),
                                        int(np.float32(g).view(np.uint32) >> 16) & 1))
        got = oracle.bf16_bits_to_double(oracle.round_bf16_bits(v, orc), orc)
        assert got == math.copysign(best, v), (v, got, best)


def test_round_bf16_double_rounding_case(orc):
    # 1 + 2^-8 + 2^-30: nearest bfloat16 is 1 + 2^-7 (above the tie); rounding through
    # float first would give the tie 1 + 2^-8 exactly, then round to even (1.0).
    v = 1.0 + 2.0 ** -8 + 2.0 ** -30
    assert oracle.bf16_bits_to_double(oracle.round_bf16_bits(v, orc), orc) == 1.0 + 2.0 ** -7
    assert oracle.round_f32(v, orc) == np.float32(v)


# ------------------------------------------------------------------ PageRank

def test_pagerank_dense_power_iteration(orc):
    rows, cols = synth.rmat(6, 4, seed=3)
    n = 1 << 6
    rp, co, _ = oracle.coo_to_csr(n, n, rows, cols, None, 0, orc)
    x = oracle.pagerank(rp, co, 0.85, 20, orc)
    A = _dense(n, n, rp, co, None)
    deg = A.sum(axis=0)
    # Google matrix written densely: columns of P are A's columns / outdeg, dangling -> 1/n
    G = np.where(deg > 0, A / np.where(deg > 0, deg, 1), 1.0 / n)
    z = np.full(n, 1.0 / n)
    for _ in range(20):
        z = 0.85 * (G @ z) + 0.15 / n
    np.testing.assert_allclose(x, z, rtol=1e-12, atol=1e-15)
    assert abs(x.sum() - 1.0) < 1e-12


# ------------------------------------------------------------------ planted mistakes

def test_planted_transposed_hilbert_fails_figure(orc):
    """A transposed curve (a plausible orientation slip) does not match the figure."""
    tabs = hilbert_figure_tables()
    bad = oracle.hilbert_table(2, orc).T
    assert not np.array_equal(bad, tabs[2])
    # a curve with the top-right quadrant merely translated (missing anti-transpose)
    good = oracle.hilbert_table(3, orc)
    bad = good.copy()
    bad[0:4, 4:8] = 48 + good[4:8, 0:4] - 16      # reuse BL quadrant's local order
    assert not np.array_equal(bad, tabs[3])


def test_planted_dropped_term_fails_brute_force(orc):
    m, n = 20, 20
    rp, co, vo = _random_csr(m, n, 80, 3, integer=True)
    x = synth.vector(n, 4, integer=True)
    y = oracle.csr_spmv(rp, co, vo, x, orc)
    bad_rp = rp.copy()
    i = int(np.argmax(np.diff(rp)))
    bad_rp[i + 1:] -= 0            # same structure ...
    bad_vo = vo.copy()
    bad_vo[rp[i]] = 0.0            # ... one term dropped
    ybad = oracle.csr_spmv(bad_rp, co, bad_vo, x, orc)
    D = _dense(m, n, rp, co, vo)
    assert np.array_equal(y, D @ x) and not np.array_equal(ybad, D @ x) or x[co[rp[i]]] == 0


def test_planted_wrong_tie_rule_fails_merge_figure(orc):
    """Consuming B first on ties would move the path; the figure's nodes catch it."""
    A, B, _, nodes, _ = _read_merge_fixture()
    i = j = 0
    walk = [(0, 0)]
    for _ in range(len(A) + len(B)):
        if i < len(A) and (j >= len(B) or A[i] < B[j]):   # strict: ties to B
            i += 1
        else:
            j += 1
        walk.append((i, j))
    assert walk != nodes


def test_csr_spmm_matches_dense_brute_force():
    """Multiple right-hand sides (Section 3): Y = A X against a dense product written out
    element by element, with integer data so that every sum is exact."""
    rng = np.random.Generator(np.random.PCG64(5))
    m, n, k = 23, 17, 5
    dense = np.where(rng.random((m, n)) < 0.3, rng.integers(-8, 9, (m, n)), 0).astype(np.float64)
    dense[4] = 0.0                                    # an empty row
    r, c = np.nonzero(dense)
    rp, co, vo = oracle.coo_to_csr(m, n, r.astype(np.int32), c.astype(np.int32), dense[r, c])
    X = rng.integers(-8, 9, (n, k)).astype(np.float64)
    Y = oracle.csr_spmm(rp, co, vo, X)
    want = np.zeros((m, k))
    for i in range(m):
        for j in range(n):
            for q in range(k):
                want[i, q] += dense[i, j] * X[j, q]
    assert Y.shape == (m, k)
    assert np.array_equal(Y, want)



# ------------------------------------------------------------------ tolerance scale (|A| |x|)

@pytest.mark.parametrize("seed", range(8))
def test_csr_absmul_dense_brute_force(orc, seed):
    """(|A| |x|)_i, the scale of every floating-point tolerance of the parity tests, against
    a dense product of the absolute values written out element by element.  Values and x
    carry mixed signs; integer data makes every sum exact, so the comparison is exact, and a
    stray term (a nonzero of the next row, a doubled entry) or a lost absolute value shows."""
    rng = np.random.default_rng(700 + seed)
    m, n = int(rng.integers(1, 48)), int(rng.integers(1, 48))
    rp, co, vo = _random_csr(m, n, int(rng.integers(0, 4 * m + 1)), 700 + seed, integer=True)
    x = synth.vector(n, 701 + seed, integer=True)
    assert (vo < 0).any() or vo.size < 4           # mixed signs present
    D = _dense(m, n, rp, co, vo)
    want = np.zeros(m)
    for i in range(m):
        for j in range(n):
            want[i] += abs(D[i, j]) * abs(x[j])
    np.testing.assert_array_equal(oracle.csr_absmul(rp, co, vo, x, orc), want)
    # pattern matrix: |1| |x_j| summed over the row's columns
    Dp = _dense(m, n, rp, co, None)
    np.testing.assert_array_equal(oracle.csr_absmul(rp, co, None, x, orc), Dp @ np.abs(x))


def test_csr_absmul_float_bounds(orc):
    """Floating values: the row sum of |a||x| equals math.fsum of the same products within
    the row length's rounding bound, and is never below the magnitude of Algorithm 1's y."""
    rp, co, vo = _random_csr(30, 30, 200, 71)
    x = synth.vector(30, 72)
    s = oracle.csr_absmul(rp, co, vo, x, orc)
    y = oracle.csr_spmv(rp, co, vo, x, orc)
    for i in range(30):
        terms = [abs(float(vo[k])) * abs(float(x[co[k]])) for k in range(rp[i], rp[i + 1])]
        L = len(terms)
        assert abs(s[i] - math.fsum(terms)) <= 2 * L * 2.0 ** -53 * math.fsum(terms)
        assert abs(y[i]) <= s[i] * (1 + 4 * L * 2.0 ** -53)


def test_planted_absmul_row_overrun_fails_brute_force(orc):
    """Summing one entry past each row's end (an off-by-one in the row loop) inflates the
    tolerance scale; the dense pin catches it."""
    m, n = 12, 12
    rp, co, vo = _random_csr(m, n, 60, 73, integer=True)
    x = synth.vector(n, 74, integer=True)
    good = oracle.csr_absmul(rp, co, vo, x, orc)
    bad_rp = rp.copy()
    bad_rp[1:-1] += 1                  # every row but the last reaches into the next one
    bad = oracle.csr_absmul(bad_rp, co, vo, x, orc)
    D = _dense(m, n, rp, co, vo)
    want = np.abs(D) @ np.abs(x)
    assert np.array_equal(good, want) and not np.array_equal(bad, want)


# ------------------------------------------------------------------ conjugate gradients

def _spd(n, nnz, seed):
    """B + B^T + D with D the row sums of |B + B^T| plus one: strictly diagonally dominant with a
    positive diagonal, hence symmetric positive definite (triplets, duplicates summed)."""
    r, c = synth.random_coo(n, n, nnz, seed)
    v = synth.values(r, c, seed)
    rows = np.concatenate([r, c]).astype(np.int32)
    cols = np.concatenate([c, r]).astype(np.int32)
    vals = np.concatenate([v, v])
    dense = np.zeros((n, n))
    np.add.at(dense, (rows, cols), vals)
    d = np.abs(dense).sum(axis=1) + 1.0
    rows = np.concatenate([rows, np.arange(n, dtype=np.int32)])
    cols = np.concatenate([cols, np.arange(n, dtype=np.int32)])
    vals = np.concatenate([vals, d])
    return rows, cols, vals, dense + np.diag(d)


@pytest.mark.parametrize("seed", range(4))
def test_cg_matches_dense_solve(orc, seed):
    """CG on a small SPD matrix reaches the dense solution (numpy.linalg.solve) and stops
    within n iterations (exact arithmetic would terminate in at most n)."""
    n = 40
    rows, cols, vals, D = _spd(n, 120, 300 + seed)
    rp, co, vo = oracle.coo_to_csr(n, n, rows, cols, vals, 0, orc)
    b = synth.vector(n, 301 + seed)
    x, it, res = oracle.cg(rp, co, vo, b, tol=1e-13, max_iters=4 * n, lib=orc)
    xs = np.linalg.solve(D, b)
    assert it <= n
    assert np.max(np.abs(x - xs)) <= 1e-10 * np.max(np.abs(xs))
    assert np.linalg.norm(b - D @ x) <= 1e-11 * np.linalg.norm(b)


def test_planted_cg_sign_error_fails_the_dense_solve(orc):
    """CG with the residual update sign flipped (r += alpha q) does not reach the solution."""
    n = 30
    rows, cols, vals, D = _spd(n, 90, 310)
    b = synth.vector(n, 311)
    x = np.zeros(n); r = b.copy(); p = b.copy(); rho = r @ r
    for _ in range(2 * n):
        q = D @ p
        alpha = rho / (p @ q)
        x = x + alpha * p
        r = r + alpha * q                     # planted mistake
        rho1 = r @ r
        p = r + (rho1 / rho) * p
        rho = rho1
    assert not np.allclose(x, np.linalg.solve(D, b), rtol=1e-6)


# ------------------------------------------------------------------ CSB / CSBH (Sections 3.1, 4.1)

@pytest.mark.parametrize("inner", [0, 1, 2])
def test_csb_structure_and_round_trip(orc, inner):
    """Row-major block order; inside a block Z-Morton (2), the block's own Hilbert curve (0) or
    rows (1), checked against the figure-pinned curve indices entry by entry, and the round
    trip back to CRS is exact."""
    m, n, lb = 50, 37, 3
    rp, co, vo = _random_csr(m, n, 400, 19)
    b = oracle.csr_to_hb(m, n, rp, co, vo, lb, inner, orc, block_order=1)
    K = oracle.grid_order(m, n, orc)
    bcols = 1 << (K - lb)
    ent = []
    for t in range(b["nblk"]):
        for k in range(b["blk_ptr"][t], b["blk_ptr"][t + 1]):
            ri, ci = int(b["idx"][k]) >> 16, int(b["idx"][k]) & 0xFFFF
            ent.append((int(b["blk_row"][t]), int(b["blk_col"][t]), ri, ci, b["val"][k]))
    blocks = [(br, bc) for br, bc, *_ in ent]
    assert [br * bcols + bc for br, bc in blocks] == sorted(br * bcols + bc for br, bc in blocks)
    for t in range(b["nblk"]):
        seq = ent[b["blk_ptr"][t]:b["blk_ptr"][t + 1]]
        if inner == 2:
            keys = [oracle.zmorton_table(lb, orc)[ri, ci] for _, _, ri, ci, _ in seq]
        elif inner == 0:
            keys = [oracle.hilbert_table(lb, orc)[ri, ci] for _, _, ri, ci, _ in seq]
        else:
            keys = [ri * (1 << lb) + ci for _, _, ri, ci, _ in seq]
        assert keys == sorted(keys) and len(set(keys)) == len(keys)
    D = np.zeros((m, n))
    for br, bc, ri, ci, v in ent:
        D[br * (1 << lb) + ri, bc * (1 << lb) + ci] += v
    np.testing.assert_array_equal(D, _dense(m, n, rp, co, vo))


def test_zmorton_block_order_matches_figure(orc):
    """Z-Morton inside a 4x4 block reproduces the paper's Z-Morton figure order."""
    from conftest import golden_path  # noqa: F401
    tab = oracle.zmorton_table(2, orc)
    order = [tuple(np.argwhere(tab == i)[0]) for i in range(16)]
    assert order[:8] == [(0, 0), (0, 1), (1, 0), (1, 1), (0, 2), (0, 3), (1, 2), (1, 3)]


# ------------------------------------------------------------------ Merge Blocking (Section 4.3)

def _nonempty_blocks(D, lb):
    """Block rows and columns of the non-empty beta x beta blocks of a dense matrix, row-major."""
    m, n = D.shape
    b = 1 << lb
    out = []
    for br in range((m + b - 1) // b):
        for bc in range((n + b - 1) // b):
            if np.any(D[br * b:(br + 1) * b, bc * b:(bc + 1) * b] != 0):
                out.append((br, bc))
    return out


@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_mergeb_block_crs_matches_dense_blocks(orc, seed, inner):
    """The CRS over blocks: blocks of block row i are ptr[i]..ptr[i+1]-1, in the order and number
    of the non-empty blocks of the dense matrix (nonzero values, so a stored entry is a dense
    nonzero)."""
    rng = np.random.default_rng(100 + seed)
    m, n = int(rng.integers(1, 60)), int(rng.integers(1, 60))
    r, c = synth.random_coo(m, n, int(rng.integers(0, 5 * m + 1)), seed)
    v = np.abs(synth.values(r, c, seed, integer=True)) + 1.0
    rp, co, vo = oracle.coo_to_csr(m, n, r, c, v, 0, orc)
    for lb in [1, 2, 3]:
        mb = oracle.csr_to_mergeb(m, n, rp, co, vo, lb, inner, orc)
        lbe = mb["log2beta"]
        D = _dense(m, n, rp, co, vo)
        want = _nonempty_blocks(D, lbe)
        got = [(int(mb["blk_row"][k]), int(mb["blk_col"][k])) for k in range(mb["nblk"])]
        assert got == want
        ptr = mb["blk_row_ptr"]
        assert len(ptr) == mb["nbr"] + 1 == (m + (1 << lbe) - 1 >> lbe) + 1
        assert ptr[0] == 0 and ptr[-1] == mb["nblk"] and (np.diff(ptr) >= 0).all()
        for i in range(mb["nbr"]):
            assert ptr[i + 1] - ptr[i] == sum(1 for br, _ in want if br == i)
            assert all(int(mb["blk_row"][k]) == i for k in range(ptr[i], ptr[i + 1]))


@pytest.mark.parametrize("inner", [0, 1])
@pytest.mark.parametrize("parts", [1, 2, 3, 7, 64, 100000])
def test_mergeb_spmv_integer_equals_dense(orc, parts, inner):
    """Integer data: every part count (down to one path item per part) gives D @ x exactly;
    carries of block rows split over several parts are added back."""
    rows, cols = synth.rmat(8, 8, seed=5)
    m = n = 1 << 8
    vals = synth.values(rows, cols, 5, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    x = synth.vector(n, 6, integer=True)
    D = _dense(m, n, rp, co, vo)
    for lb in [2, 4, 6]:
        mb = oracle.csr_to_mergeb(m, n, rp, co, vo, lb, inner, orc)
        np.testing.assert_array_equal(oracle.mergeb_spmv(m, mb, x, parts, orc), D @ x)


@pytest.mark.parametrize("shape", [(1, 1), (1, 40), (40, 1), (37, 53), (53, 37), (3, 300)])
def test_mergeb_spmv_ragged_shapes(orc, shape):
    """Non-square, partial last block row and column, a single row, pattern data."""
    m, n = shape
    rp, co, vo = _random_csr(m, n, 3 * max(m, n), 8, integer=True)
    x = synth.vector(n, 9, integer=True)
    D = _dense(m, n, rp, co, vo)
    for lb in [1, 3, 5]:
        for inner in (0, 1):
            mb = oracle.csr_to_mergeb(m, n, rp, co, vo, lb, inner, orc)
            for parts in (1, 4, 29):
                np.testing.assert_array_equal(oracle.mergeb_spmv(m, mb, x, parts, orc), D @ x)
            pat = dict(mb, val=None)
            np.testing.assert_array_equal(oracle.mergeb_spmv(m, pat, x, 3, orc), _dense(m, n, rp, co, None) @ x)


def test_mergeb_spmv_float_within_summation_order(orc):
    rows, cols = synth.rmat(9, 8, seed=3)
    m = n = 1 << 9
    vals = synth.values(rows, cols, 3)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    x = synth.vector(n, 4)
    ref = oracle.csr_spmv(rp, co, vo, x, orc)
    scale = oracle.csr_absmul(rp, co, vo, x, orc)
    for inner in (0, 1):
        mb = oracle.csr_to_mergeb(m, n, rp, co, vo, 5, inner, orc)
        y = oracle.mergeb_spmv(m, mb, x, 13, orc)
        assert (np.abs(y - ref) <= 1e-13 * scale).all()


def test_planted_mergeb_carry_overwrite_fails_dense(orc):
    """Writing a part's carry over y instead of adding it (a plausible slip in the fix-up)
    breaks the dense product as soon as a block row is split between parts."""
    rows, cols = synth.rmat(8, 8, seed=5)
    m = n = 1 << 8
    vals = synth.values(rows, cols, 5, integer=True)
    rp, co, vo = oracle.coo_to_csr(m, n, rows, cols, vals, 0, orc)
    x = synth.vector(n, 6, integer=True)
    mb = oracle.csr_to_mergeb(m, n, rp, co, vo, 5, 1, orc)
    beta, nbr, parts = 1 << mb["log2beta"], mb["nbr"], 7
    # the same walk as the oracle, written here with the carry stored instead of added
    ptr, bp, bc, idx, val = mb["blk_row_ptr"], mb["blk_ptr"], mb["blk_col"], mb["idx"], mb["val"]
    total = nbr + mb["nblk"]
    L = -(-total // parts)
    y = np.zeros(m)
    carries = []
    for p in range(parts):
        i, b = oracle.merge_path_search(min(p * L, total), ptr, orc)
        i1, b1 = oracle.merge_path_search(min((p + 1) * L, total), ptr, orc)
        temp = np.zeros(beta)
        while i < i1 or b < b1:
            if i < i1 and ptr[i + 1] <= b:
                y[i * beta:min(m, (i + 1) * beta)] = temp[:min(m, (i + 1) * beta) - i * beta]
                temp[:] = 0
                i += 1
            else:
                for t in range(bp[b], bp[b + 1]):
                    temp[int(idx[t]) >> 16] += val[t] * x[(int(bc[b]) << mb["log2beta"]) + (int(idx[t]) & 0xFFFF)]
                b += 1
        carries.append((i, temp.copy()))
    for i, temp in carries:
        if i < nbr:
            y[i * beta:min(m, (i + 1) * beta)] = temp[:min(m, (i + 1) * beta) - i * beta]   # planted
    D = _dense(m, n, rp, co, vo)
    np.testing.assert_array_equal(oracle.mergeb_spmv(m, mb, x, parts, orc), D @ x)
    assert not np.array_equal(y, D @ x)
