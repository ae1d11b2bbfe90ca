"""Wide blocks on the GPU (l = 9 .. 128 columns, rows of 16 .. 128 floats) against the float64
oracle: orthogonal iteration ("PM k Vectors" with l = k), Rayleigh-Ritz ("k Eigenvectors"), and
k-means on wide embeddings (Sec. 2.2, Sec. 4's comparison variants at the configurations' k).

Bars as for l <= 8: the orthonormal basis within 1e-5 relative Frobenius of the oracle's (the
unique basis with positive-diagonal R); Ritz values within 1e-5 of a dense eigendecomposition;
k-means++ picks identical unless a draw lies within the documented error window of a boundary,
labels identical except near-ties (margin < 1e-6), iterations and inertia equal when the labels
are; ARI of the GPU pipeline at least the oracle pipeline's minus 0.01.
"""
import numpy as np
import pytest

import workloads as W
from _helpers import fixed_point_scales, near_boundary, rel_fro, require_cuda
from oracle import kmeans as km
from oracle import metrics, omp, spectral
from oracle.rng import gaussian_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return require_cuda()


@pytest.mark.parametrize("l,every", [(12, 1), (12, 4), (20, 4), (40, 4), (100, 4)])
def test_wide_orthogonal_iteration_matches_oracle(torch, l, every):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([400] * 12, 0.05, 0.003, l)
    G = fsc.Graph.from_workload(g)
    t, seed = 10, 3 + l
    emb = fsc.embed_orthogonal(G, l, t, seed, every=every).cpu().numpy()
    assert emb.shape[1] == fsc.pad_l(l) and np.all(emb[:, l:] == 0)
    emb = emb[:, :l].astype(np.float64)
    ref = spectral.orthogonal_iteration(g, l, t, every, seed)
    err = rel_fro(emb, ref)
    print(f"orthogonal iteration l={l} every={every}: relative error {err:.2e}")
    assert err <= 1e-5, err
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    Q = emb / dm
    assert np.allclose(Q.T @ Q, np.eye(l), atol=5e-5)


def test_wide_orthogonal_iteration_weighted_and_t0(torch):
    """A weighted graph (the kNN mixture) and t = 0 (the orthonormal start block)."""
    import paper_2310_10939_gb300 as fsc
    g = W.knn_mixture(3000, 8, 5, 10, seed=6)
    G = fsc.Graph.from_workload(g)
    emb = fsc.embed_orthogonal(G, 24, 8, 7, every=2).cpu().numpy()[:, :24].astype(np.float64)
    assert rel_fro(emb, spectral.orthogonal_iteration(g, 24, 8, 2, 7)) <= 1e-5
    emb0 = fsc.embed_orthogonal(G, 17, 0, 8).cpu().numpy()[:, :17].astype(np.float64)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    assert rel_fro(emb0, dm * spectral.orthonormal_basis(gaussian_block(g.n, 17, 8))) <= 1e-5


@pytest.mark.parametrize("l", [12, 33])
def test_wide_ritz_pairs_match_dense_eigenpairs(torch, l):
    """Rayleigh-Ritz on the wide basis: values against a dense float64 eigendecomposition of M on a
    graph with a clear gap after the l-th eigenvalue (l planted blocks), and against the oracle's
    Ritz values on the same basis."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([12] * l, 0.9, 0.004, l)
    G = fsc.Graph.from_workload(g)
    vals, emb = fsc.top_eigenvectors(G, l, 200, 17, every=5)
    w, V = np.linalg.eigh(spectral.dense_signless(g))
    order = np.argsort(-w)[:l]
    assert np.allclose(vals, w[order], atol=1e-5)
    ref_vals, _ = spectral.ritz_vectors(g, l, 200, 5, 17)
    assert np.allclose(vals, ref_vals, atol=1e-5)
    dm = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    Q = emb.cpu().numpy()[:, :l].astype(np.float64) / dm
    P = V[:, order] @ V[:, order].T                      # the top-l eigenspace
    assert rel_fro(P @ Q, Q) <= 1e-3
    assert np.allclose(Q.T @ Q, np.eye(l), atol=1e-4)


def _mixture(n, k, l, seed, lp):
    rng = np.random.default_rng(seed)
    centres = rng.normal(0, 3, size=(k, l))
    X = np.zeros((n, lp), dtype=np.float32)
    X[:, :l] = centres[rng.integers(0, k, n)] + rng.normal(0, 0.5, size=(n, l))
    return X


def _kmeans_parity(torch, X, l, k, seed, ref):
    import paper_2310_10939_gb300 as fsc
    n, lp = X.shape
    lab, st, cen, sd = fsc.kmeans(torch.as_tensor(X, device="cuda"), l, k, seed, want_centroids=True, want_seeds=True)
    lab, sd = lab.cpu().numpy(), sd.cpu().numpy()
    if not np.array_equal(sd, ref["seeds"]):
        assert near_boundary(X[:, :l], k, seed, ref["seeds"]), (sd, ref["seeds"])
        return None
    margin = km.relative_margin(ref["best"], ref["second"])
    diff = lab != ref["labels"]
    assert not (diff & (margin >= 1e-6)).any(), int((diff & (margin >= 1e-6)).sum())
    if not diff.any():
        assert st["iterations"] == ref["iters"]
        assert np.isclose(st["inertia"], ref["inertia"], rtol=1e-6)
        Sx, _ = fixed_point_scales(X[:, :l], n, l)
        assert np.allclose(cen.cpu().numpy(), ref["centroids"][:, :l], rtol=1e-12, atol=2.0 ** -Sx + 1e-15)
    assert st["device_status"] == 0
    return lab


@pytest.mark.parametrize("n,k,l", [(6000, 10, 10), (8000, 16, 16), (5000, 12, 30), (4000, 20, 50), (3000, 7, 128)])
def test_wide_kmeans_matches_oracle(torch, n, k, l):
    import paper_2310_10939_gb300 as fsc
    lp = fsc.pad_l(l)
    X = _mixture(n, k, l, seed=n + l, lp=lp)
    ref = km.kmeans(X[:, :l], k, seed=5 + k)
    _kmeans_parity(torch, X, l, k, 5 + k, ref)


def test_wide_kmeans_k100_l100_against_the_all_core_oracle(torch):
    """k = 100 clusters of 100-dimensional points (the 2^22-vertex configuration's k, as l = k):
    against the C restatement of the oracle (pinned to the numpy oracle on the CPU)."""
    X = _mixture(20000, 100, 100, seed=11, lp=128)
    ref = omp.kmeans(X[:, :100], 100, 31)
    _kmeans_parity(torch, X, 100, 100, 31, ref)


def test_pm_k_vectors_and_k_eigs_cluster_an_sbm_with_16_blocks(torch):
    """l = k = 16: the paper's PM k Vectors and k Eigs baselines on an SBM with 16 planted blocks."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm_by_degree(40_000, 16, 20.0, 2.0, seed=12)
    G = fsc.Graph.from_workload(g)
    k, t, seed = 16, 16, 12
    emb = fsc.embed_orthogonal(G, k, t, seed, every=4)
    lab, _, _, _ = fsc.kmeans(emb, k, k, seed)
    ref_emb = spectral.orthogonal_iteration(g, k, t, 4, seed)
    ref = km.kmeans(ref_emb.astype(np.float32), k, seed)
    a_gpu, a_ref = metrics.ari(lab.cpu().numpy(), g.labels), metrics.ari(ref["labels"], g.labels)
    assert a_gpu >= a_ref - 0.01, (a_gpu, a_ref)
    _, emb_e = fsc.top_eigenvectors(G, k, 40, seed, every=5)
    lab, _, _, _ = fsc.kmeans(emb_e, k, k, seed)
    _, ref_z = spectral.ritz_vectors(g, k, 40, 5, seed)
    ref = km.kmeans(ref_z.astype(np.float32), k, seed)
    a_gpu, a_ref = metrics.ari(lab.cpu().numpy(), g.labels), metrics.ari(ref["labels"], g.labels)
    assert a_gpu >= a_ref - 0.01, (a_gpu, a_ref)


def test_k_eigs_with_100_blocks(torch):
    """l = k = 100 on an SBM with 100 planted blocks of 600 vertices: Ritz values against the oracle's
    on its own orthogonal-iteration basis, and the clustering's ARI against the oracle pipeline's
    (all-core oracle k-means on the oracle's embedding)."""
    import paper_2310_10939_gb300 as fsc
    g = W.sbm_by_degree(60_000, 100, 30.0, 3.0, seed=21)
    G = fsc.Graph.from_workload(g)
    k, t, seed = 100, 30, 21
    vals, emb = fsc.top_eigenvectors(G, k, t, seed, every=5)
    ref_vals, ref_z = spectral.ritz_vectors(g, k, t, 5, seed)
    assert np.allclose(vals, ref_vals, atol=1e-5)
    lab, _, _, _ = fsc.kmeans(emb, k, k, seed)
    ref = omp.kmeans(ref_z.astype(np.float32), k, seed)
    a_gpu, a_ref = metrics.ari(lab.cpu().numpy(), g.labels), metrics.ari(ref["labels"], g.labels)
    assert a_gpu >= a_ref - 0.01, (a_gpu, a_ref)


def test_wide_arguments_are_checked(torch):
    import paper_2310_10939_gb300 as fsc
    g = W.sbm([50] * 4, 0.2, 0.02, 1)
    G = fsc.Graph.from_workload(g)
    with pytest.raises(fsc.FscError):
        fsc.embed_orthogonal(G, 129, 3, 1)
    with pytest.raises(fsc.FscError):
        fsc.embed(G, 12, 3, 1)                     # the plain power method stays at l <= 8
    X = torch.zeros((300, 128), dtype=torch.float32, device="cuda")
    with pytest.raises(fsc.FscError):
        fsc.kmeans(X, 100, 300, 1)                 # k * ld above 32768
