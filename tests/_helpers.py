"""Shared helpers for the GPU parity tests (test infrastructure, not product code)."""
import numpy as np

from oracle import kmeans as km
from oracle import spectral
from oracle.rng import kmeanspp_uniform


def rel_fro(a, b) -> float:
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    den = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (den if den > 0 else 1.0))


def require_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU test run without a CUDA device"
    import paper_2310_10939_gb300 as fsc
    fsc.lib()
    return torch


def oracle_embedding_f32(g, l, t, seed, lp):
    """Oracle embedding rounded to float32 and padded to lp columns (an input both sides share)."""
    B = spectral.embed(g, l, t, seed)
    out = np.zeros((g.n, lp), dtype=np.float32)
    out[:, :l] = B.astype(np.float32)
    return B, out


def fixed_point_scales(X, n, l):
    """The library's fixed-point scales (documented in the k-means kernel header)."""
    A = float(np.abs(X).max()) if X.size else 0.0
    N = max(1, int(np.ceil(np.log2(max(n, 2)))))
    Ex = (int(np.floor(np.log2(A))) + 1) if A > 0 else 0
    Ed = 2 * Ex + int(np.ceil(np.log2(l))) + 3
    return 62 - Ex - N, 62 - Ed - N


def near_boundary(X, k, seed, seeds):
    """True if some k-means++ draw lies within the documented error window of a prefix boundary:
    the GPU prefix is exact over D^2 truncated to 2^-Sd (error < n 2^-Sd), the oracle's float64
    sequential prefix has rounding error < n 2^-53 P_total.  `seeds` are the oracle's picks; up to
    the first pick where the two sides part, both drew from the same D^2."""
    n = X.shape[0]
    _, Sd = fixed_point_scales(X, n, X.shape[1])
    D2 = km.dist32(X, X[seeds[0]])
    for r in range(1, k):
        if r > 1:
            D2 = np.minimum(D2, km.dist32(X, X[seeds[r - 1]]))
        P = np.cumsum(D2.astype(np.float64))
        if P[-1] == 0:
            continue
        T = kmeanspp_uniform(seed, r) * P[-1]
        window = n * 2.0 ** -Sd + n * 2.0 ** -53 * P[-1]
        if np.min(np.abs(P - T)) <= window:
            return True
    return False
