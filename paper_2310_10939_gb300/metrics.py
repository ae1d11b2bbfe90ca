"""Host-side evaluation of a clustering against planted labels (not part of the GPU path).

ARI (adjusted Rand index, Hubert and Arabie) from the contingency table, the
accuracy measure the paper reports in Sec. 4.2.
"""
from __future__ import annotations

import numpy as np


def ari(labels, truth) -> float:
    a = np.asarray(labels, dtype=np.int64)
    b = np.asarray(truth, dtype=np.int64)
    a = np.unique(a, return_inverse=True)[1]
    b = np.unique(b, return_inverse=True)[1]
    nb = int(b.max()) + 1 if b.size else 1
    table = np.bincount(a * nb + b, minlength=(int(a.max()) + 1 if a.size else 1) * nb).astype(np.float64)

    def pairs(x):
        return float((x * (x - 1) / 2).sum())

    rows = table.reshape(-1, nb).sum(1)
    cols = table.reshape(-1, nb).sum(0)
    n = float(a.size)
    total = n * (n - 1) / 2
    if total == 0:
        return 1.0
    s_ij, s_a, s_b = pairs(table), pairs(rows), pairs(cols)
    expected = s_a * s_b / total
    maximum = 0.5 * (s_a + s_b)
    if maximum == expected:
        return 1.0
    return (s_ij - expected) / (maximum - expected)
