"""Pins of the oracle's polynomial-filter pieces (the learned-filter extension).

Chebyshev basis and moments against dense eigendecompositions; the expansion of gamma^t
against the plain power method (p(M) = M^t exactly); the quadratic loss against its
definition; the MLP backward pass against central finite differences.
"""
import numpy as np
import pytest

import workloads as W
from oracle import eig, filter as fl, spectral
from oracle.rng import gaussian_block


def test_parameter_count():
    assert fl.NPARAM == 16 * 64 + 64 + 64 * 64 + 64 + 9 * 64 + 9 == 5833


@pytest.mark.parametrize("make", [lambda: W.sbm([40] * 3, 0.4, 0.03, 1), lambda: W.cycle(30),
                                  lambda: W.image_grid(9, 11, 3, seed=2)])
def test_cheb_basis_matches_eigendecomposition(make):
    """T_j(A_hat) = F diag(cos(j arccos mu)) F^T: the recurrence equals the spectral form."""
    g = make()
    ev, F = eig.jacobi_eigh(spectral.dense_signless(g))
    mu = np.clip(2 * ev - 1, -1, 1)
    X = gaussian_block(g.n, 3, 4)
    K = fl.cheb_basis(g, X)
    for j in range(fl.DEGREE + 1):
        ref = F @ (np.cos(j * np.arccos(mu))[:, None] * (F.T @ X))
        assert np.allclose(K[j], ref, atol=1e-10 * np.abs(ref).max() + 1e-12)
    m = fl.moments(g, X)
    Xs = F.T @ X
    for j in range(1, fl.DEGREE + 1):
        assert np.isclose(m[j - 1], float((np.cos(j * np.arccos(mu))[:, None] * Xs * Xs).sum() / (X * X).sum()))


@pytest.mark.parametrize("t", [0, 1, 3, 8])
def test_power_coefficients_reproduce_the_power_method(t):
    """p(mu) = ((1 + mu)/2)^t in the Chebyshev basis gives exactly M^t X."""
    g = W.sbm([60] * 4, 0.2, 0.02, 3)
    X = gaussian_block(g.n, 2, 5)
    c = fl.power_coefficients(t)
    K = fl.cheb_basis(g, X)
    Y = sum(cj * Kj for cj, Kj in zip(c, K))
    ref = spectral.power_method(spectral.signless_laplacian(g), X, t)
    assert np.allclose(Y, ref, rtol=0, atol=1e-12 * np.abs(ref).max())


def test_chebyshev_product_identity_gives_moments():
    """mu_{2j} = 2<T_j, T_j> - mu_0 and mu_{2j+1} = 2<T_{j+1}, T_j> - mu_1 (T_a T_b = (T_{a+b} + T_|a-b|)/2)."""
    g = W.knn_mixture(300, 5, 3, 8, seed=1)
    X = gaussian_block(g.n, 4, 2)
    K = fl.cheb_basis(g, X, 8)
    den = (X * X).sum()
    m = fl.moments(g, X)
    mu1 = m[0]
    for j in range(1, 5):
        assert np.isclose(2 * (K[j] * K[j]).sum() / den - 1.0, m[2 * j - 1], atol=1e-12)
        assert np.isclose(2 * (K[j] * K[j - 1]).sum() / den - mu1, m[2 * j - 2], atol=1e-12)


def test_target_loss_equals_definition():
    g = W.sbm([50] * 3, 0.3, 0.02, 4)
    X = gaussian_block(g.n, 2, 6)
    G, b, e0 = fl.target(g, 3, X)
    c = np.random.default_rng(0).normal(size=9)
    K = fl.cheb_basis(g, X)
    PX = fl.top_projection(g, 3, X)
    direct = ((sum(cj * Kj for cj, Kj in zip(c, K)) - PX) ** 2).sum() / (PX ** 2).sum()
    assert np.isclose(fl.filter_loss(c, G, b, e0), direct, rtol=1e-10)
    # the projector agrees with the dense eigendecomposition
    ev, F = eig.jacobi_eigh(spectral.dense_signless(g))
    P = spectral.top_projector(ev, F, 3)
    assert np.allclose(PX, P @ X, atol=1e-8)


def test_mlp_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    theta = rng.normal(0, 0.2, fl.NPARAM)
    F = rng.normal(size=(5, 16))
    G = np.stack([np.eye(9) + 0.1 * np.outer(v, v) for v in rng.normal(size=(5, 9))])
    b = rng.normal(size=(5, 9))
    e0 = rng.uniform(1, 2, 5)
    loss, grad = fl.batch_loss_and_grad(theta, F, G, b, e0)
    idx = rng.choice(fl.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        tp = theta.copy()
        tp[i] += h
        tm = theta.copy()
        tm[i] -= h
        fd = (fl.batch_loss_and_grad(tp, F, G, b, e0)[0] - fl.batch_loss_and_grad(tm, F, G, b, e0)[0]) / (2 * h)
        assert abs(fd - grad[i]) <= 1e-6 * max(1.0, abs(fd)), i


def test_gelu_definition():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 2.0])
    from scipy.special import erf
    c, cache = fl.mlp_forward(np.zeros(fl.NPARAM), np.zeros((1, 16)))
    assert np.allclose(c, 0)
    assert np.allclose(x * fl._phi(x), 0.5 * x * (1 + erf(x / np.sqrt(2))))


def test_scalar_features_on_a_star_with_isolated_vertices():
    """Hand-computed features f[0..7] of a star K_{1,4} plus two isolated vertices (n = 7, degrees
    4, 1, 1, 1, 1, 0, 0; mean 8/7; population variance 20/7 - 64/49 = 76/49), k = 2, l = 3."""
    g = W.with_isolated(W.from_edges(5, [0, 0, 0, 0], [1, 2, 3, 4]), 2)
    X = gaussian_block(g.n, 3, 1)
    f = fl.features(g, 2, 3, X)
    expect = [np.log(7.0), np.log(8.0 / 7.0), np.sqrt(76.0) / 8.0, np.log(3.5), np.log(2.0), np.log(3.5),
              3.0 / 8.0, 2.0 / 7.0]
    assert np.allclose(f[:8], expect, rtol=1e-14, atol=1e-15), (f[:8], expect)


def test_scalar_features_on_a_cycle():
    """C_10 (every degree 2), k = 4, l = 8: f = log 10, log 2, 0, 0, log 4, log 2.5, 1, 0."""
    g = W.cycle(10)
    X = gaussian_block(g.n, 8, 2)
    f = fl.features(g, 4, 8, X)
    assert np.allclose(f[:8], [np.log(10.0), np.log(2.0), 0.0, 0.0, np.log(4.0), np.log(2.5), 1.0, 0.0],
                       rtol=1e-14, atol=1e-15)
