"""Pins of the oracle's k-means pieces (Sec. 2.2) and clustering metrics (Sec. 4.2)."""
import itertools

import numpy as np
import pytest
from scipy import stats

from oracle import kmeans as km
from oracle import metrics
from oracle.rng import kmeanspp_uniform


def _blobs(n, k, l, seed, spread=0.3):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0, 3, size=(k, l))
    lab = rng.integers(0, k, n)
    return (centres[lab] + rng.normal(0, spread, size=(n, l))).astype(np.float32), lab


def test_cost_equals_frobenius_identity():
    """COST_B = ||B - X X^T B||_F^2 (the identity used for Lemma 3.3)."""
    rng = np.random.default_rng(0)
    for _ in range(5):
        B = rng.normal(size=(80, 4))
        lab = rng.integers(0, 5, 80)
        assert np.isclose(km.cost(B, lab), metrics.cost_frobenius(B, lab), rtol=1e-12)


def test_cost_matches_definition_loops():
    rng = np.random.default_rng(1)
    B = rng.normal(size=(12, 3))
    lab = rng.integers(0, 3, 12)
    total = 0.0
    for j in set(lab.tolist()):
        pts = [B[u] for u in range(12) if lab[u] == j]
        mu = sum(pts) / len(pts)
        total += sum(float(((p - mu) ** 2).sum()) for p in pts)
    assert np.isclose(km.cost(B, lab), total, rtol=1e-14)


def test_dist32_matches_scalar_float32_order():
    X, _ = _blobs(50, 3, 5, 2)
    c = X[7] + np.float32(0.125)
    out = km.dist32(X, c)
    for i in range(50):
        acc = np.float32(0.0)
        for j in range(5):
            d = np.float32(X[i, j] - c[j])
            acc = np.float32(acc + np.float32(d * d))
        assert out[i] == acc


def test_lloyd_fixed_point_properties():
    X, _ = _blobs(400, 4, 3, 3)
    out = km.kmeans(X, 4, seed=5)
    assert out["changed"] == 0
    lab = out["labels"]
    X64 = X.astype(np.float64)
    for j in range(4):
        if (lab == j).any():
            assert np.allclose(out["centroids"][j], X64[lab == j].mean(0), rtol=1e-12)
    D = np.stack([((X64 - c) ** 2).sum(1) for c in out["centroids"].astype(np.float32)], 1)
    assert (D[np.arange(400), lab] <= D.min(1) * (1 + 1e-5) + 1e-12).all()
    assert np.isclose(out["inertia"], km.cost(X, lab), rtol=1e-5)


@pytest.mark.parametrize("n,k,seed", [(7, 2, 0), (9, 3, 1), (10, 3, 2), (8, 2, 3)])
def test_lloyd_cost_not_below_brute_force_optimum(n, k, seed):
    X, _ = _blobs(n, k, 2, seed, spread=1.0)
    best = min(km.cost(X, np.array(lab))
               for lab in itertools.product(range(k), repeat=n) if len(set(lab)) == k)
    out = km.kmeans(X, k, seed)
    assert km.cost(X, out["labels"]) >= best - 1e-9
    # Lloyd ends at a local optimum that beats a random partition
    assert km.cost(X, out["labels"]) <= km.cost(X, np.arange(n) % k) + 1e-9


def test_kmeanspp_second_centre_distribution():
    """D^2 sampling: P(second centre = i) = D2_i / sum D2 given the first centre."""
    X = np.array([[0, 0], [1, 0], [0, 2], [3, 3], [-1, 0.5], [2, -2]], dtype=np.float32)
    counts = {}
    firsts = {}
    trials = 3000
    for s in range(trials):
        idx = km.kmeanspp(X, 2, s)
        firsts.setdefault(int(idx[0]), []).append(int(idx[1]))
    for f, seconds in firsts.items():
        if len(seconds) < 300:
            continue
        d2 = km.dist32(X, X[f]).astype(np.float64)
        p = d2 / d2.sum()
        obs = np.bincount(seconds, minlength=6)
        assert obs[f] == 0
        mask = p > 0
        chi = stats.chisquare(obs[mask], p[mask] * len(seconds))
        assert chi.pvalue > 1e-4
    # first centre is uniform over the points
    firstc = np.array([len(v) for _, v in sorted(firsts.items())])
    assert stats.chisquare(firstc).pvalue > 1e-4


def test_kmeanspp_first_index_rule_and_degenerate_case():
    X = np.zeros((10, 2), dtype=np.float32)
    idx = km.kmeanspp(X, 4, seed=8)
    first = int(np.floor(kmeanspp_uniform(8, 0) * 10))
    rest = [i for i in range(10) if i != first][:3]
    assert idx.tolist() == [first] + rest


def test_ari_pair_counting_and_invariances():
    rng = np.random.default_rng(4)
    for _ in range(10):
        a = rng.integers(0, 4, 60)
        b = rng.integers(0, 3, 60)
        assert np.isclose(metrics.ari(a, b), metrics.ari_pairs(a, b), atol=1e-12)
    a = rng.integers(0, 5, 100)
    perm = rng.permutation(5)
    assert metrics.ari(a, perm[a]) == 1.0
    assert np.isclose(metrics.nmi(a, perm[a]), 1.0)


def test_ari_nmi_match_library():
    skm = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(5)
    for _ in range(5):
        a = rng.integers(0, 6, 300)
        b = np.where(rng.random(300) < 0.7, a, rng.integers(0, 6, 300))
        assert np.isclose(metrics.ari(a, b), skm.adjusted_rand_score(a, b), atol=1e-12)
        assert np.isclose(metrics.nmi(a, b), skm.normalized_mutual_info_score(a, b), atol=1e-12)


def test_misclassified_volume_brute_force():
    rng = np.random.default_rng(6)
    planted = np.repeat(np.arange(3), 10)
    lab = planted.copy()
    lab[rng.choice(30, 5, replace=False)] = rng.integers(0, 3, 5)
    lab = np.array([2, 0, 1])[lab]
    d = rng.uniform(1, 3, 30)
    brute = min(sum(d[(lab == i) != (planted == p[i])].sum() for i in range(3))
                for p in itertools.permutations(range(3)))
    assert np.isclose(metrics.misclassified_volume(lab, planted, d), brute)
    assert metrics.misclassified_volume(planted, planted, d) == 0.0


def test_kmeans_restarts_reach_the_brute_force_optimum():
    """Restarts keep the lowest-inertia run: on tiny instances where a single k-means++ + Lloyd
    run stops in a local optimum, 30 restarts reach the brute-force optimum, and restarts are
    never worse than the single run (a restart rule that kept the worst run fails here)."""
    stuck = 0
    for seed in range(12):
        X, _ = _blobs(9, 3, 2, seed, spread=1.5)
        best = min(km.cost(X, np.array(lab))
                   for lab in itertools.product(range(3), repeat=9) if len(set(lab)) == 3)
        single = km.kmeans(X, 3, seed)
        out = km.kmeans_best(X, 3, seed, n_init=30)
        assert km.cost(X, out["labels"]) <= km.cost(X, single["labels"]) + 1e-9
        if km.cost(X, single["labels"]) > best + 1e-6:
            stuck += 1
            assert abs(km.cost(X, out["labels"]) - best) <= 1e-6 * max(1.0, best), seed
    assert stuck >= 4


def test_kmeans_best_single_run_is_kmeans():
    X, _ = _blobs(300, 5, 3, 4)
    a = km.kmeans(X, 5, 11)
    b = km.kmeans_best(X, 5, 11, n_init=1)
    assert np.array_equal(a["labels"], b["labels"]) and b["run"] == 0 and a["inertia"] == b["inertia"]
