"""k-means cost, k-means++ seeding and Lloyd's algorithm (Sec. 2.2).

Inputs are float32 point sets (the embedding as the CUDA path stores it).
Decisions that turn floating point into integers are taken in float32 with a
fixed operation order, the same precision the kernels use:

  dist32(x, c) = (((0 + (x_0-c_0)^2) + (x_1-c_1)^2) + ...)   each op rounded
                 to float32 (no fused multiply-add), columns 0..l-1 in order.

Sums that feed centroids and totals are float64.

Readings of what the paper leaves open (it cites k-means++ with Lloyd and uses
a library k-means in its experiments):
  * one k-means++ candidate per round, one run (no restarts);
  * first centre: index floor(u_0 * n); round r >= 1: the smallest i whose
    float64 prefix sum of D^2 exceeds u_r * sum(D^2); if that sum is 0, the
    lowest index not chosen yet; if rounding leaves no prefix above the target,
    the largest index with D^2 > 0;
  * Lloyd: ties go to the lowest centroid index, an empty cluster keeps its
    previous centroid, stop when no label changes or after ``max_iter``
    assignment steps; centroids are float64 means, used in float32.
"""
from __future__ import annotations

import numpy as np

from .rng import kmeanspp_uniform


def cost(B: np.ndarray, labels: np.ndarray, k: int | None = None) -> float:
    """COST_B(A_1..A_k) = sum_i sum_{u in A_i} ||B(u,:) - mu_i||^2 (float64)."""
    B = np.asarray(B, dtype=np.float64)
    labels = np.asarray(labels)
    total = 0.0
    for j in np.unique(labels):
        P = B[labels == j]
        mu = P.mean(0)
        total += float(((P - mu) ** 2).sum())
    return total


def dist32(X: np.ndarray, c: np.ndarray) -> np.ndarray:
    """Squared distances of every row of X to c, float32, fixed order (module doc)."""
    X = np.asarray(X, dtype=np.float32)
    c = np.asarray(c, dtype=np.float32)
    acc = np.zeros(X.shape[0], dtype=np.float32)
    for j in range(X.shape[1]):
        d = X[:, j] - c[j]
        acc = acc + d * d
    return acc


def kmeanspp(X: np.ndarray, k: int, seed: int) -> np.ndarray:
    """k-means++ seeding (D^2 sampling) with the Philox uniforms of ``seed``."""
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    if not 1 <= k <= n:
        raise ValueError("need 1 <= k <= n")
    first = int(np.floor(kmeanspp_uniform(seed, 0) * n))
    chosen = [min(first, n - 1)]
    D2 = dist32(X, X[chosen[0]])
    for r in range(1, k):
        if r > 1:
            D2 = np.minimum(D2, dist32(X, X[chosen[r - 1]]))
        prefix = np.cumsum(D2.astype(np.float64))     # sequential, index order
        total = prefix[-1]
        if total == 0.0:
            taken = set(chosen)
            nxt = next(i for i in range(n) if i not in taken)
        else:
            target = kmeanspp_uniform(seed, r) * total
            above = np.nonzero(prefix > target)[0]
            nxt = int(above[0]) if above.size else int(np.nonzero(D2 > 0)[0][-1])
        chosen.append(nxt)
    return np.asarray(chosen, dtype=np.int64)


def assign32(X: np.ndarray, c32: np.ndarray):
    """Nearest centroid (ties -> lowest index), best and second-best float32 distances."""
    D = np.stack([dist32(X, c32[j]) for j in range(c32.shape[0])], axis=1)
    lab = np.argmin(D, axis=1)                       # first minimum = lowest index
    best = D[np.arange(D.shape[0]), lab]
    if D.shape[1] > 1:
        D2 = D.copy()
        D2[np.arange(D.shape[0]), lab] = np.inf
        second = D2.min(1)
    else:
        second = np.full_like(best, np.inf)
    return lab.astype(np.int32), best, second


def lloyd(X: np.ndarray, init_idx: np.ndarray, max_iter: int = 100):
    """Lloyd iterations from the centres X[init_idx].

    Returns dict(labels, centroids (float64), iters, inertia, changed, best, second),
    where ``inertia`` is the float64 sum of the last assignment's float32 distances.
    """
    X = np.asarray(X, dtype=np.float32)
    X64 = X.astype(np.float64)
    k = len(init_idx)
    c64 = X64[np.asarray(init_idx)].copy()
    c32 = c64.astype(np.float32)
    labels = np.full(X.shape[0], -1, dtype=np.int32)
    it = 0
    changed = X.shape[0]
    best = second = None
    inertia = 0.0
    for it in range(1, max_iter + 1):
        new, best, second = assign32(X, c32)
        changed = int((new != labels).sum())
        labels = new
        inertia = float(best.astype(np.float64).sum())
        for j in range(k):
            members = labels == j
            cnt = int(members.sum())
            if cnt > 0:
                c64[j] = X64[members].sum(0) / cnt
                c32[j] = c64[j].astype(np.float32)
        if changed == 0:
            break
    return {"labels": labels, "centroids": c64, "iters": it, "inertia": inertia,
            "changed": changed, "best": best, "second": second}


def kmeans(X: np.ndarray, k: int, seed: int, max_iter: int = 100):
    """k-means++ seeding followed by Lloyd; also returns the seed indices."""
    idx = kmeanspp(X, k, seed)
    out = lloyd(X, idx, max_iter)
    out["seeds"] = idx
    return out


def kmeans_best(X: np.ndarray, k: int, seed: int, n_init: int, max_iter: int = 100):
    """Restarts: runs r = 0..n_init-1 each seeded with seed + r (their own k-means++ draws), and
    keeps the run of lowest inertia (ties: the lowest r).  Returns that run's result plus
    `run` (its index) and `inertias` (every run's)."""
    runs = [kmeans(X, k, seed + r, max_iter) for r in range(n_init)]
    inertias = np.array([r["inertia"] for r in runs])
    best = int(np.argmin(inertias))        # first minimum = lowest run index among ties
    out = dict(runs[best])
    out["run"] = best
    out["inertias"] = inertias
    return out


def relative_margin(best: np.ndarray, second: np.ndarray) -> np.ndarray:
    """(d2 - d1) / d1 per point (inf where d1 = 0 < d2)."""
    b = best.astype(np.float64)
    s = second.astype(np.float64)
    with np.errstate(divide="ignore", invalid="ignore"):
        m = np.where(b > 0, (s - b) / b, np.where(s > b, np.inf, 0.0))
    return m
