"""Input generators: determinism, shapes and distributions of the synthetic workloads."""
import numpy as np
import pytest

import oracle
import synth


def test_rmat_deterministic_and_deduplicated():
    r1, c1 = synth.rmat(12, 8, seed=5)
    r2, c2 = synth.rmat(12, 8, seed=5)
    np.testing.assert_array_equal(r1, r2)
    np.testing.assert_array_equal(c1, c2)
    key = r1.astype(np.int64) << 12 | c1
    assert np.unique(key).size == key.size
    assert r1.max() < 4096 and c1.max() < 4096 and r1.min() >= 0
    # Graph500 skew: P(row bit = 0) = a + b = 0.76 at every level
    assert abs(np.mean((r1 >> 11) & 1 == 0) - 0.76) < 0.02
    # thread count does not change the result
    lib = synth._load()
    lib.synth_set_threads(1)
    r3, c3 = synth.rmat(12, 8, seed=5)
    lib.synth_set_threads(0)
    np.testing.assert_array_equal(r1, r3)
    np.testing.assert_array_equal(c1, c3)


def test_values_are_functions_of_position():
    r, c = synth.rmat(10, 8, seed=1)
    v = synth.values(r, c, 3)
    perm = synth.shuffle_order(r.size)
    np.testing.assert_array_equal(synth.values(r[perm], c[perm], 3), v[perm])
    assert v.min() >= -1 and v.max() < 1
    vi = synth.values(r, c, 3, integer=True)
    assert set(np.unique(vi)) <= set(range(-8, 9)) and np.all(vi == np.round(vi))


def test_erdos_renyi_and_zipf():
    r, c = synth.erdos_renyi(1000, 8, seed=2)
    assert r.size == 8000
    for i in range(0, 1000, 97):
        row = c[r == i]
        assert row.size == 8 and np.unique(row).size == 8
    r, c = synth.zipf_rows(5000, 1.8, 1 << 10, 0.05, seed=4)
    lens = np.bincount(r, minlength=5000)
    assert 0.03 < np.mean(lens == 0) < 0.08
    assert lens.max() <= 1 << 10
    key = r.astype(np.int64) * 5000 + c
    assert np.unique(key).size == key.size


def test_round_bf16_bits_matches_oracle_rounding():
    rng = np.random.default_rng(0)
    v = np.concatenate([rng.uniform(-1, 1, 4000), [0.0, -0.0, 1.0 + 2 ** -8, 1.0 + 2 ** -8 + 2 ** -30, 3.0]])
    bits = synth.round_bf16_bits(v)
    ref = np.array([oracle.round_bf16_bits(x) for x in v], np.uint16)
    np.testing.assert_array_equal(bits, ref)


def test_poisson_arrivals_and_mix():
    t = synth.poisson_arrivals(1000.0, 20000, seed=3)
    assert np.all(np.diff(t) >= 0)
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert abs(gaps.mean() - 1e-3) < 3e-5                    # mean inter-arrival 1/rate
    assert abs(gaps.std() - 1e-3) < 5e-5                     # exponential: sd = mean
    assert np.array_equal(t, synth.poisson_arrivals(1000.0, 20000, seed=3))
    kind, mat = synth.request_mix(20000, 7, 0.2, seed=3)
    assert abs(kind.mean() - 0.2) < 0.02 and set(np.unique(mat)) == set(range(7))


def test_rmat_raw_dedup_is_rmat():
    """The raw edge list, reduced to the first occurrence of every (row, col), in edge order,
    is synth.rmat's output."""
    r, c = synth.rmat_raw(11, 16, seed=5)
    key = r.astype(np.int64) << 32 | c.astype(np.int64)
    _, first = np.unique(key, return_index=True)
    first.sort()
    r2, c2 = synth.rmat(11, 16, seed=5)
    assert np.array_equal(r[first], r2) and np.array_equal(c[first], c2)


@pytest.mark.gpu
def test_gpu_generator_matches_host_bit_for_bit():
    """The GPU twin draws the same edges and values as the host generator."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    for scale, ef, seed in [(12, 16, 0), (9, 8, 77)]:
        rd, cd = synth.gpu_rmat_raw(scale, ef, seed, device="cuda:0")
        r, c = synth.rmat_raw(scale, ef, seed)
        assert np.array_equal(rd.cpu().numpy(), r) and np.array_equal(cd.cpu().numpy(), c)
        for integer in (False, True):
            v = synth.values(r, c, seed, integer=integer)
            assert np.array_equal(synth.gpu_values(rd, cd, seed, integer=integer).cpu().numpy(), v)
            assert np.array_equal(synth.gpu_values(rd, cd, seed, integer=integer, f32=True).cpu().numpy(),
                                  v.astype(np.float32))
