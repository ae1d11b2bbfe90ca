"""Pins of the oracle's random numbers (Philox4x64-10, Box-Muller, Lemma A.1)."""
import numpy as np
import pytest
from scipy import stats

from oracle import rng


@pytest.mark.parametrize("key", [(0, 0), (5, 1), (0xDEADBEEFCAFEF00D, 2), (2**64 - 1, 2**64 - 1)])
@pytest.mark.parametrize("start", [0, 1, 12345, 2**40])
def test_philox_matches_numpy_library(key, start):
    """numpy.random.Philox is Philox4x64-10; it pre-increments its counter."""
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                          counter=np.array([start, 0, 0, 0], dtype=np.uint64))
    ref = bg.random_raw(4 * 5)
    ctr = np.arange(start + 1, start + 6, dtype=np.uint64)
    w = rng.philox4x64_10(ctr, 0, 0, 0, key[0], key[1])
    mine = np.stack(w, 1).reshape(-1)
    assert np.array_equal(mine, ref)


def test_philox_high_counter_words_match_numpy():
    bg = np.random.Philox(key=np.array([7, 9], dtype=np.uint64),
                          counter=np.array([2**64 - 1, 3, 0, 11], dtype=np.uint64))
    ref = bg.random_raw(4)          # counter wraps word 0 and carries into word 1
    w = rng.philox4x64_10(np.uint64(0), np.uint64(4), np.uint64(0), np.uint64(11), 7, 9)
    assert np.array_equal(np.array([x for x in w]).reshape(-1), ref)


def test_uniform_maps_are_exact_and_in_range():
    words = np.array([0, 2**64 - 1, 2**40 - 1, 2**40, 2**63], dtype=np.uint64)
    u = rng.u24(words)
    assert (u > 0).all() and (u <= 1).all()
    assert np.array_equal(u.astype(np.float32).astype(np.float64), u)
    v = rng.u53(words)
    assert (v >= 0).all() and (v < 1).all()
    assert v[0] == 0.0 and v[1] == 1.0 - 2.0 ** -53


def test_gaussian_moments_and_normality():
    z = rng.gaussian_block(100_000, 4, seed=11).ravel()
    N = z.size
    assert abs(z.mean()) < 5 / np.sqrt(N)
    assert abs(z.var() - 1.0) < 5 * np.sqrt(2.0 / N)
    assert abs(stats.kurtosis(z, fisher=False) - 3.0) < 5 * np.sqrt(24.0 / N)
    assert stats.kstest(z, "norm").pvalue > 1e-4


def test_gaussian_columns_do_not_depend_on_l():
    a = rng.gaussian_block(1001, 2, seed=3)
    b = rng.gaussian_block(1001, 5, seed=3)
    assert np.array_equal(a, b[:, :2])
    c = rng.gaussian_block(1001, 2, seed=4)
    assert not np.allclose(a, c)


def test_gaussian_layout_matches_definition():
    """Element (i, c) comes from Philox block (c*n+i)//4, Box-Muller slot (c*n+i)%4."""
    n, l, seed = 7, 3, 99
    z = rng.gaussian_block(n, l, seed)
    for i in range(n):
        for c in range(l):
            e = c * n + i
            w = rng.philox4x64_10(np.uint64(e // 4), 0, 0, 0, seed, rng.STREAM_X0)
            j = e % 4
            p = j // 2
            u1 = float(rng.u24(w[2 * p]))
            u2 = float(rng.u24(w[2 * p + 1]))
            r = np.sqrt(-2.0 * np.log(u1))
            expect = r * (np.cos(2 * np.pi * u2) if j % 2 == 0 else np.sin(2 * np.pi * u2))
            assert z[i, c] == expect


def test_lemma_a1_chi_square_lengths():
    """Lemma A.1: ||x||^2 ~ chi^2_n and ||P x||^2 ~ chi^2_k for a rank-k projector P."""
    n, k, trials = 400, 5, 400
    X = rng.gaussian_block(n, trials, seed=21)
    sq = (X * X).sum(0)
    assert abs(sq.mean() - n) < 5 * np.sqrt(2 * n / trials)
    Q, _ = np.linalg.qr(np.random.default_rng(0).normal(size=(n, k)))
    pk = ((Q.T @ X) ** 2).sum(0)
    assert abs(pk.mean() - k) < 5 * np.sqrt(2 * k / trials)
    assert stats.kstest(pk, stats.chi2(k).cdf).pvalue > 1e-4
    # the Chebyshev bounds of the lemma hold with room to spare
    assert (pk <= 6 * k).mean() >= 1 - 1 / (25 * k) - 0.02
    assert (sq <= 6 * n).all()


def test_kmeanspp_uniform_stream_is_separate():
    a = [rng.kmeanspp_uniform(5, r) for r in range(4)]
    assert len(set(a)) == 4 and all(0 <= x < 1 for x in a)
    w = rng.philox4x64_10(np.uint64(0), 0, 0, 0, 5, rng.STREAM_X0)
    assert float(rng.u53(w[0])) != a[0]
