"""Pins of Algorithm 2 end to end (Theorem 3.2, Sec. 4.1) and planted-mistake checks."""
import numpy as np
import pytest

import workloads as W
from oracle import cluster, eig, kmeans as km, metrics, spectral


def test_pb_cliques_exact_recovery():
    """Theorem 3.2 with rho(k) = 0: k disjoint cliques are recovered exactly."""
    g = W.disjoint_cliques(6, 15)
    for seed in range(5):
        out = cluster.fast_spectral_cluster(g, 6, 3, 20, seed)
        assert metrics.ari(out["labels"], g.labels) == 1.0


def test_pg_sbm_recovery_config_small():
    """SBM n=1000, k=4, p=0.1, q=0.002, l=2, t=20: the planted partition is recovered
    (Sec. 4.1 reports recovery of the ground truth on SBM); median ARI over 10 seeds."""
    aris = []
    for seed in range(1, 11):
        g = W.sbm([250] * 4, 0.1, 0.002, seed)
        out = cluster.fast_spectral_cluster(g, 4, 2, 20, seed)
        aris.append(metrics.ari(out["labels"], g.labels))
        d = spectral.degrees(g)
        if aris[-1] == 1.0:
            assert metrics.misclassified_volume(out["labels"], g.labels, d) == 0.0
    assert np.median(aris) >= 0.99


def test_default_params():
    assert cluster.default_params(2 ** 20, 16) == (4, 20)
    assert cluster.default_params(1000, 4) == (2, 10)
    assert cluster.default_params(154401, 8) == (3, 18)
    assert cluster.paper_remark_params(1000, 4) == (2, 56)


# ---- planted mistakes: each plausible error in the oracle fails a pin -------------

def _cliques_closed_form_holds(embed_fn) -> bool:
    k, s = 3, 6
    g = W.disjoint_cliques(k, s)
    X = np.random.default_rng(0).normal(size=(g.n, 2))
    c = (s - 2) / (2 * (s - 1))
    P = np.kron(np.eye(k), np.full((s, s), 1.0 / s))
    t = 5
    B = embed_fn(g, X, t)
    expect = (P @ X + c ** t * (X - P @ X)) / np.sqrt(s - 1)
    return bool(np.allclose(B, expect, atol=1e-12))


def _correct_embed(g, X, t):
    return spectral.embed(g, X.shape[1], t, 0, x0=X)


def _eigenvalue_one_holds() -> bool:
    """P-a on a non-regular graph: M D^1/2 1 = D^1/2 1 and M symmetric."""
    g = W.sbm([30, 50], 0.3, 0.05, 2)
    M = spectral.signless_laplacian(g)
    v = np.sqrt(spectral.degrees(g))
    return bool(np.linalg.norm(M @ v - v) <= 1e-12 * np.linalg.norm(v) and abs(M - M.T).max() <= 1e-15)


def _some_pin_fails() -> bool:
    return not (_cliques_closed_form_holds(_correct_embed) and _eigenvalue_one_holds())


def test_planted_mistakes_fail_the_clique_pin(monkeypatch):
    assert not _some_pin_fails()
    mutants = {
        "drop the 1/2": lambda g: (spectral.sp.identity(g.n) - spectral.normalised_laplacian(g)).tocsr(),
        "use N instead of M": lambda g: spectral.normalised_laplacian(g),
        "D^-1 instead of D^-1/2": lambda g: (spectral.sp.identity(g.n) - 0.5 * (
            spectral.sp.diags(1 / spectral.degrees(g)) @ spectral.laplacian(g))).tocsr(),
    }
    for name, mutant in mutants.items():
        monkeypatch.setattr(spectral, "signless_laplacian", mutant)
        assert _some_pin_fails(), name
        monkeypatch.undo()
    # forgetting the final D^-1/2 scaling of Algorithm 2
    monkeypatch.setattr(spectral, "inv_sqrt_degrees", lambda d: np.ones_like(d))
    assert _some_pin_fails()


def test_planted_mistake_in_distance_fails_fixed_point_pin(monkeypatch):
    rng = np.random.default_rng(3)
    centres = np.array([[0.0, 0.0], [0.0, 3.0], [0.0, 6.0], [0.0, 9.0]])   # differ in the last coordinate only
    X = (centres[rng.integers(0, 4, 200)] + rng.normal(0, .3, (200, 2))).astype(np.float32)
    real = km.dist32

    def wrong(Xa, c):       # drops the last coordinate
        return real(np.asarray(Xa)[:, :-1], np.asarray(c)[:-1])

    monkeypatch.setattr(km, "dist32", wrong)
    out = km.kmeans(X, 4, 1)
    X64 = X.astype(np.float64)
    D = np.stack([((X64 - c) ** 2).sum(1) for c in out["centroids"]], 1)
    assert not (D[np.arange(200), out["labels"]] <= D.min(1) * (1 + 1e-5)).all()


def test_planted_transposed_eigvecs_fail_spectral_formula():
    g = W.sbm([20] * 3, 0.5, 0.05, 4)
    ev, F = eig.jacobi_eigh(spectral.dense_signless(g))
    X0 = np.random.default_rng(1).normal(size=(g.n, 2))
    Xt = spectral.power_method(spectral.signless_laplacian(g), X0, 4)
    assert np.allclose(Xt, spectral.spectral_power(ev, F, X0, 4), atol=1e-12)
    assert not np.allclose(Xt, spectral.spectral_power(ev, F.T, X0, 4), atol=1e-6)
