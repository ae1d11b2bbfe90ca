"""Pins of the oracle's operators and power method (Sec. 2, Sec. 3.1, Algorithm 1).

P-a  M D^1/2 1 = D^1/2 1 (eigenvalue 1), symmetry, spectrum in [0, 1].
P-b  disjoint cliques: closed-form spectrum and M^t X.
P-c  cycle and complete graph: closed-form spectra.
P-d  dense eigendecomposition: x_t = sum a_i gamma_i^t f_i and the
     deterministic inequality chain in the proof of Lemma 3.1.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eig, spectral
from oracle.rng import gaussian_block


def _small_weighted(n=40, seed=0):
    rng = np.random.default_rng(seed)
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(iu.size) < 0.2
    w = rng.uniform(0.1, 2.0, keep.sum())
    return W.from_edges(n, iu[keep], ju[keep], w)


def test_degree_matches_brute_force():
    g = _small_weighted()
    dense = np.zeros((g.n, g.n))
    for i in range(g.n):
        for e in range(g.row_ptr[i], g.row_ptr[i + 1]):
            dense[i, g.col[e]] = g.w[e]
    brute = [sum(dense[u, v] for u in range(g.n) if u != v) for v in range(g.n)]
    assert np.allclose(spectral.degrees(g), brute, rtol=1e-15, atol=0)


def test_laplacians_match_dense_definitions():
    g = _small_weighted(30, 1)
    A = spectral.adjacency(g).toarray()
    d = A.sum(1) - np.diag(A)
    L = np.diag(d) - A
    Dm = np.diag(1 / np.sqrt(d))
    N = Dm @ L @ Dm
    M = np.eye(g.n) - 0.5 * N
    assert np.allclose(spectral.normalised_laplacian(g).toarray(), N, atol=1e-14)
    assert np.allclose(spectral.signless_laplacian(g).toarray(), M, atol=1e-14)
    # M = (I + D^-1/2 A D^-1/2) / 2
    assert np.allclose(M, 0.5 * (np.eye(g.n) + Dm @ A @ Dm), atol=1e-14)


@pytest.mark.parametrize("make", [
    lambda: W.sbm([250] * 4, 0.1, 0.002, 1),
    lambda: _small_weighted(60, 2),
    lambda: W.image_grid(24, 31, 4, seed=1),
    lambda: W.knn_mixture(500, 8, 4, 10, seed=2),
])
def test_pa_eigenvalue_one(make):
    """P-a: D^1/2 1 is an eigenvector of M with eigenvalue 1; M symmetric, contractive."""
    g = make()
    M = spectral.signless_laplacian(g)
    v = np.sqrt(spectral.degrees(g))
    assert np.linalg.norm(M @ v - v) <= 1e-13 * np.linalg.norm(v)
    assert abs(M - M.T).max() <= 1e-15
    x = gaussian_block(g.n, 3, 5)
    assert (np.linalg.norm(M @ x, axis=0) <= np.linalg.norm(x, axis=0) * (1 + 1e-14)).all()


@pytest.mark.parametrize("k,s", [(3, 5), (4, 8)])
def test_pb_cliques_closed_form(k, s):
    """P-b: spectrum of k disjoint K_s is 1 (x k) and (s-2)/(2(s-1)) (x k(s-1));
    M^t X = P X + c^t (I - P) X with P the within-clique averaging projector."""
    g = W.disjoint_cliques(k, s)
    M = spectral.dense_signless(g)
    ev, _ = eig.jacobi_eigh(M)
    c = (s - 2) / (2 * (s - 1))
    expect = np.sort(np.concatenate([np.ones(k), np.full(k * (s - 1), c)]))
    assert np.allclose(ev, expect, atol=1e-12)
    X = gaussian_block(g.n, 3, 7)
    P = np.kron(np.eye(k), np.full((s, s), 1.0 / s))
    for t in (0, 1, 5, 20):
        Xt = spectral.power_method(spectral.signless_laplacian(g), X, t)
        assert np.allclose(Xt, P @ X + c ** t * (X - P @ X), rtol=0, atol=1e-13)
    # D^-1/2 P X is constant on each clique: the clique mean of X / sqrt(s - 1)
    B = spectral.embed(g, 3, 60, 7, x0=X)
    means = (P @ X) / np.sqrt(s - 1)
    assert np.allclose(B, means, atol=1e-12)


@pytest.mark.parametrize("n", [3, 8, 25])
def test_pc_cycle_spectrum(n):
    g = W.cycle(n)
    ev, _ = eig.jacobi_eigh(spectral.dense_signless(g))
    expect = np.sort(np.cos(np.pi * np.arange(n) / n) ** 2)
    assert np.allclose(ev, expect, atol=1e-12)
    # cosine modes are eigenvectors: M v = cos^2(pi j / n) v
    M = spectral.signless_laplacian(g)
    for j in range(n):
        v = np.cos(2 * np.pi * j * np.arange(n) / n)
        assert np.allclose(M @ v, np.cos(np.pi * j / n) ** 2 * v, atol=1e-13)


@pytest.mark.parametrize("n", [2, 5, 30])
def test_pc_complete_spectrum(n):
    g = W.complete(n)
    ev, _ = eig.jacobi_eigh(spectral.dense_signless(g))
    expect = np.sort(np.concatenate([[1.0], np.full(n - 1, (n - 2) / (2 * (n - 1)))]))
    assert np.allclose(ev, expect, atol=1e-12)


@pytest.mark.parametrize("n,seed", [(20, 0), (60, 1), (150, 2)])
def test_jacobi_matches_library_eigh(n, seed):
    S = np.random.default_rng(seed).normal(size=(n, n))
    S = S + S.T
    ev, V = eig.jacobi_eigh(S)
    ref = np.linalg.eigh(S)[0]
    assert np.allclose(ev, ref, atol=1e-10 * np.abs(ref).max())
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.allclose(S @ V, V * ev, atol=1e-12 * np.abs(ref).max())


@pytest.mark.parametrize("make,k", [
    (lambda: W.sbm([40] * 4, 0.5, 0.02, 3), 4),
    (lambda: W.image_grid(10, 14, 3, seed=4), 3),
    (lambda: W.knn_mixture(180, 6, 3, 8, seed=5), 3),
])
def test_pd_dense_spectral_formula_and_lemma31_chain(make, k):
    """P-d: x_t = sum a_i gamma_i^t f_i; and for every column,
    ||x_t - P x_0|| <= (1 - gamma_k^t) ||P x_0|| + gamma_{k+1}^t ||x_0||."""
    g = make()
    M = spectral.dense_signless(g)
    ev, F = eig.jacobi_eigh(M)
    assert ev.min() >= -1e-12 and ev.max() <= 1 + 1e-12
    X0 = gaussian_block(g.n, 4, 9)
    gam = np.sort(ev)[::-1]
    P = spectral.top_projector(ev, F, k)
    for t in (1, 7, 20):
        Xt = spectral.power_method(spectral.signless_laplacian(g), X0, t)
        Xs = spectral.spectral_power(ev, F, X0, t)
        assert np.linalg.norm(Xt - Xs) <= 1e-11 * np.linalg.norm(Xs)
        lhs = np.linalg.norm(Xt - P @ X0, axis=0)
        rhs = (1 - gam[k - 1] ** t) * np.linalg.norm(P @ X0, axis=0) + gam[k] ** t * np.linalg.norm(X0, axis=0)
        assert (lhs <= rhs * (1 + 1e-10) + 1e-12).all()


def test_isolated_vertex_reading():
    g = W.with_isolated(W.sbm([30] * 2, 0.4, 0.05, 1), 3)
    M = spectral.signless_laplacian(g).toarray()
    for v in range(g.n - 3, g.n):
        e = np.zeros(g.n)
        e[v] = 1
        assert np.array_equal(M[v], e)
    B = spectral.embed(g, 2, 10, 1)
    assert np.array_equal(B[-3:], np.zeros((3, 2)))


def test_power_method_t0_is_identity_and_embed_scales():
    g = W.sbm([25] * 2, 0.4, 0.05, 2)
    X = gaussian_block(g.n, 2, 1)
    assert np.array_equal(spectral.power_method(spectral.signless_laplacian(g), X, 0), X)
    d = spectral.degrees(g)
    assert np.allclose(spectral.embed(g, 2, 0, 1), X / np.sqrt(d)[:, None], rtol=1e-15)


def test_orthogonal_iteration_spans_the_power_method_block():
    """Orthonormalising never changes the span, so orthogonal iteration with any interval gives
    the orthonormal basis (positive-diagonal R) of M^t X0 itself: the same Q as one QR at the end."""
    g = W.sbm([40, 50, 60], 0.3, 0.02, 3)
    X0 = gaussian_block(g.n, 3, 11)
    Y = spectral.power_method(spectral.signless_laplacian(g), X0, 9)
    Q_end = spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None] * spectral.orthonormal_basis(Y)
    for every in (1, 2, 4, 9):
        Z = spectral.orthogonal_iteration(g, 3, 9, every, 11)
        assert np.allclose(Z, Q_end, atol=1e-10), every


def test_orthogonal_iteration_converges_to_the_top_eigenvectors():
    """On a graph with a clear gap after the top l eigenvalues of M, the basis converges to that
    eigenspace (dense eigendecomposition), and its columns are orthonormal in x-space."""
    g = W.sbm([60, 60, 60, 60], 0.5, 0.01, 5)
    l = 4
    Z = spectral.orthogonal_iteration(g, l, 200, 5, 2)
    Q = Z / spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    assert np.allclose(Q.T @ Q, np.eye(l), atol=1e-10)
    w, V = np.linalg.eigh(spectral.dense_signless(g))
    P = V[:, np.argsort(-w)[:l]]
    assert np.linalg.norm(P @ P.T - Q @ Q.T, 2) < 1e-6


def test_ritz_pairs_converge_to_the_top_eigenpairs():
    """Rayleigh-Ritz on the orthogonal-iteration basis recovers the top l eigenpairs of M
    (dense eigendecomposition): values to 1e-9, vectors up to sign."""
    g = W.sbm([50, 60, 70, 80], 0.4, 0.02, 7)
    l = 4
    theta, Z = spectral.ritz_vectors(g, l, 300, 10, 3)
    w, V = np.linalg.eigh(spectral.dense_signless(g))
    order = np.argsort(-w)[:l]
    assert np.allclose(theta, w[order], atol=1e-9)
    Q = Z / spectral.inv_sqrt_degrees(spectral.degrees(g))[:, None]
    for a in range(l):
        c = abs(float(Q[:, a] @ V[:, order[a]]))
        assert c > 1 - 1e-8, (a, c)
