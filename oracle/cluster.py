"""Algorithm 2 (FastSpectralCluster) end to end, in the oracle's precision.

Steps in the paper's order: M = I - N/2; l Gaussian vectors; y_i =
PowerMethod(M, x_i, t); Y = [y_1..y_l]; k-means on the rows of D^-1/2 Y.
The embedding is float64; it is rounded to float32 before k-means so that the
k-means decisions are taken in the precision of the CUDA path (see kmeans).

Parameter readings (the paper fixes l and t only up to constants, Sec. 3.2):
  default_params      l = max(1, ceil(log2 k)), t = ceil(log2 n)
  paper_remark_params l = max(1, ceil(ln k)),  t = ceil(10 ln(n / k))
                      (the "works well in practice" remark after Theorem 3.2).
"""
from __future__ import annotations

import math

import numpy as np

from . import kmeans as km
from .spectral import embed


def default_params(n: int, k: int):
    l = max(1, math.ceil(math.log2(k))) if k > 1 else 1
    t = max(0, math.ceil(math.log2(n))) if n > 1 else 0
    return l, t


def paper_remark_params(n: int, k: int):
    l = max(1, math.ceil(math.log(k))) if k > 1 else 1
    t = max(0, math.ceil(10.0 * math.log(n / k))) if n > k else 0
    return l, t


def fast_spectral_cluster(g, k: int, l: int, t: int, seed: int, max_iter: int = 100):
    """Labels of Algorithm 2 plus the float64 embedding and k-means details."""
    B = embed(g, l, t, seed)
    out = km.kmeans(B.astype(np.float32), k, seed, max_iter)
    out["embedding"] = B
    return out
