"""k-nearest-neighbour graph of a point set (the Sec. 4.2 pre-processing), plain definitions.

Test infrastructure (only tests, smoke() and bench's CPU legs use it).

The paper builds "the k nearest neighbour graph" with k = 10 and says no more; the reading taken
(shared with the CUDA library, which implements it independently):
  * distance: d2(i, j) = sum over c = 0..dim-1, in that order, of (x_i[c] - x_j[c])^2 in float32
    with no fused multiply-add (both sides then take every neighbour decision in the same
    float32 arithmetic);
  * neighbours of i: the knn points j != i of smallest d2, ties to the lower index;
  * symmetrised by union: {i, j} is an edge if j is a neighbour of i or i of j;
  * sigma: the median (mean of the two middle values for an even count) of the n * knn directed
    distances sqrt(d2) (float32 square roots);
  * weight of {i, j}: exp(-d2(i, j) / sigma^2).
"""
from __future__ import annotations

import numpy as np


def sqdist32(x: np.ndarray, ys: np.ndarray) -> np.ndarray:
    """float32 d2 from point x to each row of ys, columns summed in order (no fma)."""
    x = np.asarray(x, dtype=np.float32)
    ys = np.asarray(ys, dtype=np.float32)
    acc = np.zeros(ys.shape[0], dtype=np.float32)
    for c in range(ys.shape[1]):
        diff = (ys[:, c] - x[c]).astype(np.float32)
        acc = (acc + (diff * diff).astype(np.float32)).astype(np.float32)
    return acc


def neighbours(X: np.ndarray, knn: int):
    """(idx, d2): n x knn neighbour indices sorted by (d2, index), and their float32 d2."""
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    idx = np.empty((n, knn), dtype=np.int64)
    dd = np.empty((n, knn), dtype=np.float32)
    for i in range(n):
        d = sqdist32(X[i], X)
        d[i] = np.inf
        order = np.lexsort((np.arange(n), d))[:knn]       # by d2, then by index
        idx[i] = order
        dd[i] = d[order]
    return idx, dd


def knn_graph(X: np.ndarray, knn: int):
    """CSR (row_ptr int64, col int32 sorted per row, w float64) of the union-symmetrised kNN
    graph, sigma, and the directed neighbour lists."""
    X = np.asarray(X, dtype=np.float32)
    n = X.shape[0]
    idx, dd = neighbours(X, knn)
    dist = np.sqrt(dd).astype(np.float32).ravel()
    sigma = float(np.median(dist.astype(np.float64)))
    rows = [set() for _ in range(n)]
    for i in range(n):
        for j in idx[i]:
            rows[i].add(int(j))
            rows[int(j)].add(i)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    cols, ws = [], []
    for i in range(n):
        c = np.array(sorted(rows[i]), dtype=np.int64)
        d2 = sqdist32(X[i], X[c]).astype(np.float64)
        cols.append(c)
        ws.append(np.exp(-d2 / sigma ** 2))
        row_ptr[i + 1] = row_ptr[i] + c.size
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, dtype=np.int32)
    w = np.concatenate(ws) if ws else np.zeros(0)
    return row_ptr, col, w, sigma, idx, dd
