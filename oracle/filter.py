"""Polynomial filters p(M) = sum_j c_j T_j(2M - I), graph features and the filter MLP (float64).

Not in the paper: an extension that replaces M^t of Algorithm 2 by a degree-8 polynomial
chosen per graph.  The quantity it is judged by is the one Lemma 3.1 bounds,
||p(M) x_0 - P x_0|| with P the projector on the top-k eigenvectors of M.

Definitions used here (and restated independently by the CUDA library):
  A_hat = 2M - I = D^-1/2 A D^-1/2, eigenvalues mu = 2 gamma - 1 in [-1, 1].
  Chebyshev recurrence: T_0 x = x, T_1 x = A_hat x, T_{j+1} x = 2 A_hat T_j x - T_{j-1} x.
  Moments of a block X (n x l): mu_j = sum_c x_c^T T_j x_c / sum_c x_c^T x_c, sums over the
    vertices with d(v) > 0.
  Features (16): log n, log mean degree, degree std / mean, log(max degree / mean degree),
    log k, log(n / k), l / 8, fraction of isolated vertices, mu_1 .. mu_8 of the start block.
  Target of a graph: K_j = T_j(A_hat) X (j = 0..8), PX; G = [<K_a, K_b>], b = [<K_a, PX>],
    e0 = ||PX||^2 (Frobenius inner products); loss(c) = (c^T G c - 2 b^T c + e0) / e0
    = ||sum_j c_j K_j - PX||_F^2 / ||PX||_F^2.
  MLP: h1 = gelu(W1 f + b1) (64), h2 = gelu(W2 h1 + b2) (64), c = W3 h2 + b3 (9),
    gelu(x) = x Phi(x) with Phi the standard normal CDF; parameters flattened in the order
    W1 (64 x 16, row-major), b1, W2 (64 x 64), b2, W3 (9 x 64), b3 (5833 numbers).

Parity unpinned against the paper (the paper has no learned filter); the MLP's backward pass
is pinned by central finite differences, the basis and moments by dense eigendecompositions.
"""
from __future__ import annotations

from math import erf, exp, pi, sqrt

import numpy as np
import scipy.sparse.linalg as sla

from . import spectral

DEGREE = 8
NFEAT = 16
HIDDEN = 64
NCOEF = DEGREE + 1
SHAPES = [("W1", (HIDDEN, NFEAT)), ("b1", (HIDDEN,)), ("W2", (HIDDEN, HIDDEN)), ("b2", (HIDDEN,)),
          ("W3", (NCOEF, HIDDEN)), ("b3", (NCOEF,))]
NPARAM = sum(int(np.prod(s)) for _, s in SHAPES)


def a_hat(g):
    """D^-1/2 A D^-1/2 (sparse, float64); rows of isolated vertices are zero."""
    dm = spectral.sp.diags(spectral.inv_sqrt_degrees(spectral.degrees(g)))
    return (dm @ spectral.adjacency(g) @ dm).tocsr()


def cheb_basis(g, X: np.ndarray, degree: int = DEGREE):
    """[T_0 X, ..., T_degree X] by the three-term recurrence in A_hat."""
    A = a_hat(g)
    K = [np.array(X, dtype=np.float64)]
    if degree >= 1:
        K.append(A @ K[0])
    for _ in range(2, degree + 1):
        K.append(2.0 * (A @ K[-1]) - K[-2])
    return K


def moments(g, X: np.ndarray, degree: int = DEGREE) -> np.ndarray:
    """mu_1..mu_degree of the block X (definition in the module doc), taken over the vertices
    with d(v) > 0: an isolated vertex has no embedding coordinate (its D^-1/2 is read as 0), so
    its row of X carries no information about the graph and is left out of the moments."""
    keep = spectral.degrees(g) > 0
    K = cheb_basis(g, X, degree)
    Xk = X[keep]
    den = float((Xk * Xk).sum())
    return np.array([float((Xk * K[j][keep]).sum()) / den for j in range(1, degree + 1)])


def features(g, k: int, l: int, X: np.ndarray) -> np.ndarray:
    d = spectral.degrees(g)
    n = g.n
    mean = d.mean()
    f = np.zeros(NFEAT)
    f[0] = np.log(n)
    f[1] = np.log(mean)
    f[2] = d.std() / mean
    f[3] = np.log(d.max() / mean)
    f[4] = np.log(k)
    f[5] = np.log(n / k)
    f[6] = l / 8.0
    f[7] = float((d == 0).mean())
    f[8:] = moments(g, X)
    return f


def top_projection(g, k: int, X: np.ndarray) -> np.ndarray:
    """P X for P the projector on the k largest-eigenvalue eigenvectors of M (ARPACK)."""
    M = spectral.signless_laplacian(g)
    if k >= g.n - 1:
        w, V = np.linalg.eigh(M.toarray())
        V = V[:, np.argsort(-w)[:k]]
    else:
        w, V = sla.eigsh(M, k=k, which="LA", tol=1e-10, maxiter=100000)
    return V @ (V.T @ X)


def target(g, k: int, X: np.ndarray, degree: int = DEGREE):
    """(G, b, e0) of a graph for the quadratic filter loss."""
    K = cheb_basis(g, X, degree)
    PX = top_projection(g, k, X)
    G = np.array([[float((Ka * Kb).sum()) for Kb in K] for Ka in K])
    b = np.array([float((Ka * PX).sum()) for Ka in K])
    return G, b, float((PX * PX).sum())


def filter_loss(c, G, b, e0) -> float:
    c = np.asarray(c, dtype=np.float64)
    return float((c @ G @ c - 2.0 * b @ c + e0) / e0)


def power_coefficients(t: int, degree: int = DEGREE) -> np.ndarray:
    """Chebyshev coefficients (in mu = 2 gamma - 1) of gamma^t = ((1 + mu) / 2)^t, t <= degree."""
    from numpy.polynomial import chebyshev as C
    from numpy.polynomial import polynomial as Pn
    mono = Pn.polypow([0.5, 0.5], t)                  # ((1 + mu) / 2)^t in powers of mu
    c = C.poly2cheb(mono)
    out = np.zeros(degree + 1)
    out[:c.size] = c
    return out


# ---- the MLP in float64 with a hand-written backward pass ---------------------------------

def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in SHAPES:
        size = int(np.prod(shape))
        out[name] = np.asarray(theta[o:o + size], dtype=np.float64).reshape(shape)
        o += size
    return out


def _phi(x):
    return np.vectorize(lambda v: 0.5 * (1.0 + erf(v / sqrt(2.0))))(x)


def _pdf(x):
    return np.vectorize(lambda v: exp(-0.5 * v * v) / sqrt(2.0 * pi))(x)


def mlp_forward(theta: np.ndarray, F: np.ndarray):
    """Coefficients (B x 9) for features F (B x 16), and the cache for the backward pass."""
    p = unpack(theta)
    F = np.atleast_2d(np.asarray(F, dtype=np.float64))
    a1 = F @ p["W1"].T + p["b1"]
    h1 = a1 * _phi(a1)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = a2 * _phi(a2)
    c = h2 @ p["W3"].T + p["b3"]
    return c, (F, a1, h1, a2, h2)


def mlp_backward(theta: np.ndarray, cache, dc: np.ndarray) -> np.ndarray:
    """Gradient of sum(dc * c) w.r.t. the flattened parameters."""
    p = unpack(theta)
    F, a1, h1, a2, h2 = cache
    g = {"W3": dc.T @ h2, "b3": dc.sum(0)}
    dh2 = dc @ p["W3"]
    da2 = dh2 * (_phi(a2) + a2 * _pdf(a2))
    g["W2"] = da2.T @ h1
    g["b2"] = da2.sum(0)
    dh1 = da2 @ p["W2"]
    da1 = dh1 * (_phi(a1) + a1 * _pdf(a1))
    g["W1"] = da1.T @ F
    g["b1"] = da1.sum(0)
    return np.concatenate([g[name].reshape(-1) for name, _ in SHAPES])


def batch_loss_and_grad(theta, F, G, b, e0):
    """Mean filter loss over a batch and its gradient (float64)."""
    c, cache = mlp_forward(theta, F)
    B = c.shape[0]
    loss = 0.0
    dc = np.zeros_like(c)
    for i in range(B):
        loss += filter_loss(c[i], G[i], b[i], e0[i])
        dc[i] = (2.0 * G[i] @ c[i] - 2.0 * b[i]) / e0[i]
    return loss / B, mlp_backward(theta, cache, dc / B)
