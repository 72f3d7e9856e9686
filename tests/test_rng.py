"""The method's random draws (reading R15): the oracle's generator pinned to
published values and to the distributions it must produce, and the library's
generator (host code, callable without a GPU) bit-equal to the oracle's.

Eq. 1 wants hash vectors with N(0,1) entries and Alg. 1 a uniform sample of
the points. Both sides implement splitmix64 (Steele, Lea and Flood, OOPSLA
2014) with Box-Muller and a partial Fisher-Yates shuffle from the published
definitions, independently.
"""

import math

import numpy as np
import pytest
from scipy import stats

import paper_2406_10938_gb300 as pkg
from oracle import detlsh_oracle as O


# ------------------------------------------------------------------ oracle pins
def test_splitmix64_published_outputs():
    # the first outputs of the reference splitmix64 from state 0
    g = O.splitmix64(0)
    assert [next(g) for _ in range(5)] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F,
                                           0xF88BB8A8724C81EC, 0x1B39896A51A8749B]


def test_hash_entries_are_standard_normal():
    A = O.draw_hashes(3, 4, 16, 960).astype(np.float64).ravel()
    assert A.shape == (61_440,)
    assert abs(A.mean()) < 4.0 / math.sqrt(A.size)
    assert abs(A.var() - 1.0) < 0.03
    assert stats.kstest(A, "norm").pvalue > 1e-3
    # the cos and sin halves of each Box-Muller pair are uncorrelated
    assert abs(np.corrcoef(A[0::2], A[1::2])[0, 1]) < 0.03
    # rows are distinct draws
    assert not np.array_equal(A[:960], A[960:1920])


def test_hash_vectors_give_the_lemma1_chi2_law():
    # Lemma 1: for fixed o1, o2 and a row block of K N(0,1) vectors,
    # ||P(o1) - P(o2)||^2 / ||o1 - o2||^2 ~ chi2(K)
    K, d = 16, 24
    rng = np.random.default_rng(5)
    o = rng.standard_normal(d)
    r = []
    for seed in range(400):
        A = O.draw_hashes(seed, 1, K, d).astype(np.float64)
        r.append(float(np.sum((A @ o) ** 2) / np.sum(o ** 2)))
    assert stats.kstest(r, stats.chi2(K).cdf).pvalue > 1e-3


def test_sample_is_distinct_sorted_in_range():
    for n, n_s in ((10, 10), (10, 1), (1000, 999), (12_345, 100), (5, 3)):
        s = O.draw_sample(7, n, n_s)
        assert s.shape == (n_s,)
        assert (np.diff(s) > 0).all()
        assert s[0] >= 0 and s[-1] < n
    assert np.array_equal(O.draw_sample(1, 37, 37), np.arange(37))


def test_sample_is_uniform():
    # every id is included with probability n_s/n
    n, n_s, seeds = 40, 8, 3000
    counts = np.zeros(n)
    for seed in range(seeds):
        counts[O.draw_sample(seed, n, n_s)] += 1
    expect = seeds * n_s / n
    assert stats.chisquare(counts, np.full(n, expect)).pvalue > 1e-3
    # and every pair of ids together with probability n_s(n_s-1)/(n(n-1))
    both = sum(1 for seed in range(seeds) if {3, 29} <= set(O.draw_sample(seed, n, n_s).tolist()))
    p = n_s * (n_s - 1) / (n * (n - 1))
    assert abs(both - seeds * p) < 4 * math.sqrt(seeds * p * (1 - p))


def test_default_sample_size_is_a_tenth():
    assert [O.default_sample_size(n) for n in (1, 10, 11, 1_000_000, 99)] == [1, 1, 2, 100_000, 10]


# ------------------------------------------------------------------ library = oracle
@pytest.fixture(scope="module")
def built():
    pkg.build()
    return pkg


@pytest.mark.parametrize("seed,L,K,d", [(3, 4, 16, 128), (0, 1, 16, 960), (2**64 - 1, 3, 5, 7),
                                        (12345, 16, 16, 33), (9, 1, 1, 1)])
def test_library_hashes_equal_oracle(built, seed, L, K, d):
    got = built.detlsh_draw_hashes(seed, L * K, d).numpy()
    ref = O.draw_hashes(seed, L, K, d)
    assert got.dtype == ref.dtype
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("seed,n,n_s", [(3, 1_000_000, 10_000), (3, 1_000_000, 100_000), (5, 10_000, 1_000),
                                        (0, 100_000_000, 1_000), (11, 64, 64), (2**63, 1, 1),
                                        (17, 2**32 - 1, 257)])
def test_library_sample_equals_oracle(built, seed, n, n_s):
    got = built.detlsh_draw_sample(seed, n, n_s).numpy()
    assert np.array_equal(got, O.draw_sample(seed, n, n_s))


def test_library_draws_reject_bad_sizes(built):
    L = built.lib()
    assert L.detlsh_draw_hashes(1, 0, 4, None) == -1
    assert L.detlsh_draw_sample(1, 10, 11, None) == -1
    import ctypes
    buf = (ctypes.c_int64 * 4)()
    assert L.detlsh_draw_sample(1, 10, 0, buf) == -1
    assert L.detlsh_draw_sample(1, 2**32, 4, buf) == -1
