"""Orthogonal iteration (the power method on a D-orthonormalised block; "PM k Vectors" with l = k)
on the GPU against the float64 oracle."""
import numpy as np
import pytest

import workloads as W
from _helpers import rel_fro, require_cuda
from oracle import cluster as ocluster
from oracle import kmeans as km
from oracle import metrics, spectral
from oracle.rng import gaussian_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.mark.parametrize("every", [1, 4])
@pytest.mark.parametrize("name", ["sbm", "knn"])
def test_orthogonal_iteration_matches_oracle(torch, name, every):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([700, 800, 900, 600], 0.03, 0.002, 5) if name == "sbm" else W.knn_mixture(3000, 8, 5, 10, seed=6)
    G = fsc.Graph.from_workload(g)
    l, t, seed = (4, 12, 3) if name == "sbm" else (5, 10, 4)
    emb = fsc.embed_orthogonal(G, l, t, seed, every=every).cpu().numpy()[:, :l].astype(np.float64)
    ref = spectral.orthogonal_iteration(g, l, t, every, seed)
    print(f"orthogonal iteration {name} l={l} every={every}: relative error {rel_fro(emb, ref):.2e}")
    assert rel_fro(emb, ref) <= 1e-5
    # the same basis as one QR of M^t X0 at the end (the span never changes)
    Y = spectral.power_method(spectral.signless_laplacian(g), gaussian_block(g.n, l, seed), t)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    assert rel_fro(emb, dm * spectral.orthonormal_basis(Y)) <= 1e-5
    Q = emb / dm
    assert np.allclose(Q.T @ Q, np.eye(l), atol=2e-5)


def test_orthogonal_iteration_t0_is_the_orthonormal_start_block(torch):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([300, 400], 0.05, 0.005, 9)
    G = fsc.Graph.from_workload(g)
    emb = fsc.embed_orthogonal(G, 3, 0, 8).cpu().numpy()[:, :3].astype(np.float64)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    assert rel_fro(emb, dm * spectral.orthonormal_basis(gaussian_block(g.n, 3, 8))) <= 1e-5


def test_pm_k_vectors_clusters_an_sbm(torch):
    """l = k = 8 orthogonal vectors (the paper's PM k Vectors baseline) with the library's k-means,
    against the oracle's clustering of its own orthogonal-iteration embedding."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm_by_degree(40_000, 8, 20.0, 2.0, seed=12)
    G = fsc.Graph.from_workload(g)
    k, t, seed = 8, 16, 12
    emb = fsc.embed_orthogonal(G, k, t, seed, every=4)
    lab, st, _, _ = fsc.kmeans(emb, k, k, seed)
    ref_emb = spectral.orthogonal_iteration(g, k, t, 4, seed)
    ref = km.kmeans(ref_emb.astype(np.float32), k, seed)
    a_gpu = metrics.ari(lab.cpu().numpy(), g.labels)
    a_ref = metrics.ari(ref["labels"], g.labels)
    assert a_gpu >= a_ref - 0.01, (a_gpu, a_ref)


def test_ritz_pairs_match_dense_eigenpairs(torch):
    """Rayleigh-Ritz on the orthogonal-iteration basis: values and vectors (up to sign) against a
    dense float64 eigendecomposition of M on a graph with a clear gap."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([150, 200, 250, 300], 0.2, 0.01, 17)
    G = fsc.Graph.from_workload(g)
    l = 4
    vals, emb = fsc.top_eigenvectors(G, l, 200, 17, every=5)
    w, V = np.linalg.eigh(spectral.dense_signless(g))
    order = np.argsort(-w)[:l]
    assert np.allclose(vals, w[order], atol=1e-5)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    Q = emb.cpu().numpy()[:, :l].astype(np.float64) / dm
    for a in range(l):
        assert abs(float(Q[:, a] @ V[:, order[a]])) > 1 - 1e-3, a
    ref_vals, ref_Z = spectral.ritz_vectors(g, l, 200, 5, 17)
    assert np.allclose(vals, ref_vals, atol=1e-5)


def test_k_eigs_embedding_clusters_an_sbm(torch):
    """The paper's "k Eigs" baseline for k <= 8: k-means on the top-k Ritz vectors."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm_by_degree(30_000, 8, 20.0, 2.0, seed=23)
    G = fsc.Graph.from_workload(g)
    k = 8
    _, emb = fsc.top_eigenvectors(G, k, 60, 23, every=5)
    lab, _, _, _ = fsc.kmeans(emb, k, k, 23)
    _, ref_Z = spectral.ritz_vectors(g, k, 60, 5, 23)
    ref = km.kmeans(ref_Z.astype(np.float32), k, 23)
    a_gpu = metrics.ari(lab.cpu().numpy(), g.labels)
    a_ref = metrics.ari(ref["labels"], g.labels)
    assert a_gpu >= a_ref - 0.01, (a_gpu, a_ref)
