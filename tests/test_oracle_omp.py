"""Pins of the all-core C/OpenMP restatement of the oracle against the sequential numpy oracle.

The numpy oracle is pinned against the paper (closed forms, dense eigendecompositions, brute
force); the C restatement is timed on all host cores, so it must compute the same thing: the
same start block and k-means++ uniforms (Philox4x64-10), the same embedding to float64 rounding,
the same k-means++ picks and Lloyd labels (near-ties aside) on the same float32 points.
"""
import numpy as np
import pytest

import workloads as W
from oracle import kmeans as km
from oracle import omp, rng, spectral


def test_start_block_and_uniforms_match_the_numpy_generator():
    a = omp.gaussian_block(1001, 3, 17)
    b = rng.gaussian_block(1001, 3, 17)
    assert np.allclose(a, b, rtol=1e-14, atol=1e-14)
    assert all(omp.load().orc_kmeanspp_uniform(9, r) == rng.kmeanspp_uniform(9, r) for r in range(20))


@pytest.mark.parametrize("make,l,t", [
    (lambda: W.sbm([250] * 4, 0.1, 0.002, 3), 2, 20),
    (lambda: W.with_isolated(W.sbm([60, 80], 0.2, 0.02, 4), 3), 3, 7),
    (lambda: W.image_grid(20, 30, 4, seed=2), 4, 12),
    (lambda: W.knn_mixture(800, 6, 4, 10, seed=3), 5, 0),
])
def test_embedding_matches_the_numpy_oracle(make, l, t):
    g = make()
    csr = omp.Csr(g)
    deg, dinv = omp.degrees(csr)
    assert np.allclose(deg, spectral.degrees(g), rtol=1e-15, atol=0)
    x = omp.gaussian_block(g.n, l, 5)
    omp.power_method(csr, deg, dinv, x, t)
    ref = spectral.embed(g, l, t, 5)
    B = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None] * x
    assert np.linalg.norm(B - ref) <= 1e-13 * np.linalg.norm(ref)
    assert np.array_equal(omp.embed(g, l, t, 5), omp.embedding_f32(dinv, x))


def test_power_method_planted_slip_is_caught():
    """The pin above is strict enough: the same loop with N in place of M (a dropped 1/2) differs."""
    g = W.sbm([100] * 3, 0.1, 0.01, 1)
    csr = omp.Csr(g)
    deg, dinv = omp.degrees(csr)
    x = omp.gaussian_block(g.n, 2, 1)
    omp.power_method(csr, deg, dinv, x, 3)
    N = spectral.normalised_laplacian(g)
    y = rng.gaussian_block(g.n, 2, 1)
    for _ in range(3):
        y = N @ y
    assert np.linalg.norm(x - y) > 1e-3 * np.linalg.norm(y)


def _mixture(n, k, l, seed):
    r = np.random.default_rng(seed)
    c = r.normal(0, 3, size=(k, l))
    return (c[r.integers(0, k, n)] + r.normal(0, 0.5, size=(n, l))).astype(np.float32)


@pytest.mark.parametrize("n,k,l,seed", [(5000, 7, 3, 1), (20000, 30, 5, 2), (999, 1, 2, 3), (64, 64, 2, 4)])
def test_kmeans_matches_the_numpy_oracle(n, k, l, seed):
    X = _mixture(n, max(1, k // 2), l, seed)
    a = omp.kmeans(X, k, seed)
    b = km.kmeans(X, k, seed)
    assert np.array_equal(a["seeds"], b["seeds"])
    margin = km.relative_margin(b["best"], b["second"])
    assert not ((a["labels"] != b["labels"]) & (margin >= 1e-6)).any()
    if np.array_equal(a["labels"], b["labels"]):
        assert a["iters"] == b["iters"]
        assert np.allclose(a["centroids"], b["centroids"], rtol=1e-12, atol=1e-12)
        assert np.isclose(a["inertia"], b["inertia"], rtol=1e-12)


def test_kmeans_degenerate_identical_points():
    X = np.zeros((300, 2), dtype=np.float32)
    a = omp.kmeans(X, 4, 3)
    b = km.kmeans(X, 4, 3)
    assert np.array_equal(a["seeds"], b["seeds"]) and np.array_equal(a["labels"], b["labels"])


def test_cluster_end_to_end_matches_on_an_sbm():
    g = W.sbm([250] * 4, 0.1, 0.002, 6)
    from oracle import cluster as oc
    from oracle import metrics
    a = omp.fast_spectral_cluster(g, 4, 2, 20, 6)
    b = oc.fast_spectral_cluster(g, 4, 2, 20, 6)
    assert abs(metrics.ari(a["labels"], g.labels) - metrics.ari(b["labels"], g.labels)) <= 0.01


def test_lloyd_distances_match_the_numpy_oracle():
    """The last assignment's nearest and second-nearest distances (the margin rule's inputs)."""
    X = _mixture(3000, 6, 4, 9)
    a = omp.kmeans(X, 6, 2)
    b = km.kmeans(X, 6, 2)
    if np.array_equal(a["labels"], b["labels"]):
        assert np.array_equal(a["best"], b["best"]) and np.array_equal(a["second"], b["second"])
