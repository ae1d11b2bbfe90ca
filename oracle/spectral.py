"""Graph operators and the power-method embedding, in float64 (Sec. 2, Algorithms 1-2).

Definitions followed (Sec. 2, Preliminaries):
  d(v)  = sum over u != v of w(u, v)                       (degree)
  L     = D - A,  N = D^-1/2 L D^-1/2                       (normalised Laplacian)
  M     = I - N / 2                                         (signless Laplacian,
          eigenvalues gamma_i = 1 - lambda_i / 2 in [0, 1], same eigenvectors)
Reading for an isolated vertex v (d(v) = 0, where D^-1/2 is undefined):
  D^-1/2(v, v) := 0, so row v of N is zero, row v of M is e_v and the
  embedding row of v is zero.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .rng import gaussian_block


def _rows(g) -> np.ndarray:
    return np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr))


def _weights(g) -> np.ndarray:
    return np.ones(g.nnz, dtype=np.float64) if g.w is None else g.w.astype(np.float64)


def degrees(g) -> np.ndarray:
    """d(v) = sum_{u != v} w(u, v), float64."""
    rows = _rows(g)
    off = rows != g.col
    return np.bincount(rows[off], weights=_weights(g)[off], minlength=g.n).astype(np.float64)


def inv_sqrt_degrees(d: np.ndarray) -> np.ndarray:
    """Diagonal of D^-1/2 with the isolated-vertex reading (0 where d = 0)."""
    out = np.zeros_like(d)
    pos = d > 0
    out[pos] = 1.0 / np.sqrt(d[pos])
    return out


def adjacency(g) -> sp.csr_matrix:
    """Weighted adjacency matrix A (float64, CSR)."""
    return sp.csr_matrix((_weights(g), g.col.astype(np.int64), g.row_ptr), shape=(g.n, g.n))


def volume(d: np.ndarray, members) -> float:
    """vol(S) = sum of degrees over S."""
    return float(d[np.asarray(members)].sum())


def laplacian(g) -> sp.csr_matrix:
    """L = D - A."""
    return (sp.diags(degrees(g)) - adjacency(g)).tocsr()


def normalised_laplacian(g) -> sp.csr_matrix:
    """N = D^-1/2 L D^-1/2."""
    dm = sp.diags(inv_sqrt_degrees(degrees(g)))
    return (dm @ laplacian(g) @ dm).tocsr()


def signless_laplacian(g) -> sp.csr_matrix:
    """M = I - N / 2 (the paper's scaled signless Laplacian)."""
    return (sp.identity(g.n, format="csr") - 0.5 * normalised_laplacian(g)).tocsr()


def power_method(M, x0: np.ndarray, t: int) -> np.ndarray:
    """Algorithm 1: x_i = M x_{i-1} for i = 1..t, no normalisation; returns x_t.

    ``x0`` may be a matrix: each column is run independently (same operator).
    """
    x = np.array(x0, dtype=np.float64, copy=True)
    for _ in range(t):
        x = M @ x
    return x


def embed(g, l: int, t: int, seed: int, x0: np.ndarray | None = None) -> np.ndarray:
    """Algorithm 2 up to k-means: D^-1/2 [PowerMethod(M, x_i, t)]_{i=1..l}.

    The l start vectors are N(0, I) draws from the Philox stream of ``seed``
    unless ``x0`` (n x l) is given.
    """
    M = signless_laplacian(g)
    if x0 is None:
        x0 = gaussian_block(g.n, l, seed)
    Y = power_method(M, x0, t)
    return inv_sqrt_degrees(degrees(g))[:, None] * Y


def orthonormal_basis(Y: np.ndarray) -> np.ndarray:
    """Q with orthonormal columns and Y = Q R, R upper triangular with positive diagonal (the
    unique thin QR factor of a full-rank Y; numpy's Householder QR with the signs fixed)."""
    Q, R = np.linalg.qr(Y)
    s = np.sign(np.diag(R))
    s[s == 0] = 1.0
    return Q * s


def orthogonal_iteration(g, l: int, t: int, every: int, seed: int, x0: np.ndarray | None = None) -> np.ndarray:
    """The power method on a block of l vectors kept orthonormal (orthogonal iteration; with
    l = k it is the "PM k Vectors" variant compared in Sec. 4): Y <- M Y for t steps, Y replaced by
    its orthonormal basis (above) after every `every` steps and after the last; returns the
    embedding D^-1/2 Y (n x l)."""
    from .rng import gaussian_block
    M = signless_laplacian(g)
    Y = gaussian_block(g.n, l, seed) if x0 is None else np.array(x0, dtype=np.float64)
    for it in range(t):
        Y = M @ Y
        if (it + 1) % every == 0 or it == t - 1:
            Y = orthonormal_basis(Y)
    return inv_sqrt_degrees(degrees(g))[:, None] * Y


def ritz_vectors(g, l: int, t: int, every: int, seed: int):
    """Rayleigh-Ritz on the orthogonal-iteration basis: with Q its x-space basis (orthonormal),
    H = Q^T M Q, H = V diag(theta) V^T (theta descending); returns (theta, D^-1/2 Q V).  For t
    large enough the pairs converge to the top l eigenpairs of M (the "k Eigs" embedding of the
    paper's comparison when l = k)."""
    dm = inv_sqrt_degrees(degrees(g))[:, None]
    Q = orthogonal_iteration(g, l, t, every, seed) / np.where(dm > 0, dm, 1.0)
    H = Q.T @ (signless_laplacian(g) @ Q)
    theta, V = np.linalg.eigh(0.5 * (H + H.T))
    order = np.argsort(-theta, kind="stable")
    return theta[order], dm * (Q @ V[:, order])


def dense_signless(g) -> np.ndarray:
    """M as a dense float64 matrix (small graphs)."""
    return signless_laplacian(g).toarray()


def spectral_power(evals: np.ndarray, evecs: np.ndarray, x0: np.ndarray, t: int) -> np.ndarray:
    """x_t = sum_i a_i gamma_i^t f_i with a_i = <x_0, f_i> (Sec. 3.1), for a full eigenbasis."""
    a = evecs.T @ x0
    return evecs @ ((evals ** t)[:, None] * a)


def top_projector(evals: np.ndarray, evecs: np.ndarray, k: int) -> np.ndarray:
    """P = sum_{i<=k} f_i f_i^T over the k largest eigenvalues of M."""
    order = np.argsort(-evals, kind="stable")[:k]
    F = evecs[:, order]
    return F @ F.T
