"""Clustering quality measures used in Sec. 4 and Theorem 3.2.

ARI: adjusted Rand index (Hubert and Arabie) from the contingency table.
NMI: mutual information normalised by the arithmetic mean of the two
     entropies (a choice: the paper does not state its normalisation).
Misclassified volume: min over label permutations sigma of
     sum_i vol(A_i symdiff S_sigma(i)) (Theorem 3.2).
Frobenius cost: COST_B = ||B - X X^T B||_F^2 with X the normalised
     partition indicator (the identity used in the proof of Lemma 3.3).
"""
from __future__ import annotations

from math import comb

import numpy as np


def contingency(a, b) -> np.ndarray:
    a = np.asarray(a)
    b = np.asarray(b)
    _, ai = np.unique(a, return_inverse=True)
    _, bi = np.unique(b, return_inverse=True)
    C = np.zeros((ai.max() + 1, bi.max() + 1), dtype=np.int64)
    np.add.at(C, (ai, bi), 1)
    return C


def ari(a, b) -> float:
    """Adjusted Rand index of two labelings."""
    C = contingency(a, b)
    n = int(C.sum())
    sum_ij = sum(comb(int(x), 2) for x in C.ravel())
    sum_a = sum(comb(int(x), 2) for x in C.sum(1))
    sum_b = sum(comb(int(x), 2) for x in C.sum(0))
    total = comb(n, 2)
    if total == 0:
        return 1.0
    expected = sum_a * sum_b / total
    maximum = 0.5 * (sum_a + sum_b)
    if maximum == expected:
        return 1.0
    return float((sum_ij - expected) / (maximum - expected))


def ari_pairs(a, b) -> float:
    """ARI by explicit O(n^2) pair counting (small n; brute-force check of ari)."""
    a = np.asarray(a)
    b = np.asarray(b)
    n = a.size
    iu, ju = np.triu_indices(n, 1)
    sa = a[iu] == a[ju]
    sb = b[iu] == b[ju]
    both = int((sa & sb).sum())
    na = int(sa.sum())
    nb = int(sb.sum())
    total = iu.size
    if total == 0:
        return 1.0
    expected = na * nb / total
    maximum = 0.5 * (na + nb)
    if maximum == expected:
        return 1.0
    return float((both - expected) / (maximum - expected))


def _entropy(counts: np.ndarray) -> float:
    p = counts[counts > 0] / counts.sum()
    return float(-(p * np.log(p)).sum())


def nmi(a, b) -> float:
    """Normalised mutual information, arithmetic-mean normalisation."""
    C = contingency(a, b).astype(np.float64)
    n = C.sum()
    pij = C / n
    pi = pij.sum(1, keepdims=True)
    pj = pij.sum(0, keepdims=True)
    nz = pij > 0
    mi = float((pij[nz] * np.log(pij[nz] / (pi @ pj)[nz])).sum())
    ha = _entropy(C.sum(1))
    hb = _entropy(C.sum(0))
    if ha + hb == 0:
        return 1.0
    return 2.0 * mi / (ha + hb)


def misclassified_volume(labels, planted, d: np.ndarray) -> float:
    """min_sigma sum_i vol(A_i symdiff S_sigma(i)) via an optimal label matching."""
    from scipy.optimize import linear_sum_assignment
    labels = np.asarray(labels)
    planted = np.asarray(planted)
    ka = int(labels.max()) + 1
    ks = int(planted.max()) + 1
    k = max(ka, ks)
    V = np.zeros((k, k))
    np.add.at(V, (labels, planted), d)            # volume of A_i intersect S_j
    volA = V.sum(1)
    volS = V.sum(0)
    sym = volA[:, None] + volS[None, :] - 2.0 * V  # vol(A_i symdiff S_j)
    r, c = linear_sum_assignment(sym)
    return float(sym[r, c].sum())


def cost_frobenius(B: np.ndarray, labels) -> float:
    """||B - X X^T B||_F^2 with X(u, i) = 1/sqrt(|A_i|) for u in A_i."""
    B = np.asarray(B, dtype=np.float64)
    labels = np.asarray(labels)
    ids = np.unique(labels)
    X = np.zeros((B.shape[0], ids.size))
    for c, j in enumerate(ids):
        members = labels == j
        X[members, c] = 1.0 / np.sqrt(members.sum())
    R = B - X @ (X.T @ B)
    return float((R * R).sum())
