"""Counter-based random numbers for the oracle.

Philox4x64-10 is written from its published definition (Salmon, Moraes, Dror,
Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4-word counter
and a 2-word key, ten rounds of two 64x64->128-bit multiplications with the
key bumped by the Weyl constants between rounds.

Streams used by the method (key = (seed, stream)):
  stream 1 - the l Gaussian start vectors x_1..x_l of Algorithm 2.
  stream 2 - the uniforms of k-means++ seeding.

Gaussian layout: element (i, c) of the n x l start block has linear index
e = c * n + i (column-major, so column c is the same vector for any l >= c+1).
Philox block b = e // 4 yields four words w0..w3; element j = e % 4 uses the
Box-Muller pair (u1, u2) = (U24(w[2(j//2)]), U24(w[2(j//2)+1])) and takes the
cosine branch for even j, the sine branch for odd j, where
U24(w) = ((w >> 40) + 1) / 2^24 lies in (0, 1] and is exact in float32.
k-means++ uniforms: U53(w) = (w >> 11) / 2^53 in [0, 1), from word 0 of
counter (round, 0, 0, 0).
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1
PHILOX_M0 = 0xD2E7470EE14C6C93
PHILOX_M1 = 0xCA5A826395121157
PHILOX_W0 = 0x9E3779B97F4A7C15
PHILOX_W1 = 0xBB67AE8584CAA73B

STREAM_X0 = 1
STREAM_KMEANSPP = 2


def _mulhilo(a: np.ndarray, m: int):
    """(hi, lo) words of the 128-bit product of uint64 array ``a`` and constant ``m``."""
    a = a.astype(np.uint64)
    lo32 = np.uint64(0xFFFFFFFF)
    s32 = np.uint64(32)
    a_lo = a & lo32
    a_hi = a >> s32
    m_lo = np.uint64(m & 0xFFFFFFFF)
    m_hi = np.uint64(m >> 32)
    p_ll = a_lo * m_lo
    p_lh = a_lo * m_hi
    p_hl = a_hi * m_lo
    p_hh = a_hi * m_hi
    mid = (p_ll >> s32) + (p_lh & lo32) + (p_hl & lo32)
    hi = p_hh + (p_lh >> s32) + (p_hl >> s32) + (mid >> s32)
    lo = a * np.uint64(m)            # wraps modulo 2^64
    return hi, lo


def philox4x64_10(c0, c1, c2, c3, k0: int, k1: int):
    """Philox4x64-10 of counter words (arrays, broadcast) under key (k0, k1)."""
    c = [np.asarray(x, dtype=np.uint64) for x in np.broadcast_arrays(c0, c1, c2, c3)]
    k0 = np.uint64(k0 & MASK64)
    k1 = np.uint64(k1 & MASK64)
    with np.errstate(over="ignore"):
        for _ in range(10):
            hi0, lo0 = _mulhilo(c[0], PHILOX_M0)
            hi1, lo1 = _mulhilo(c[2], PHILOX_M1)
            c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
            k0 = np.uint64((int(k0) + PHILOX_W0) & MASK64)
            k1 = np.uint64((int(k1) + PHILOX_W1) & MASK64)
    return c


def u24(w: np.ndarray) -> np.ndarray:
    """Uniform in (0, 1] from the top 24 bits of a 64-bit word (exact in float32)."""
    return ((w >> np.uint64(40)).astype(np.float64) + 1.0) * 2.0 ** -24


def u53(w: np.ndarray) -> np.ndarray:
    """Uniform in [0, 1) from the top 53 bits of a 64-bit word (exact in float64)."""
    return (w >> np.uint64(11)).astype(np.float64) * 2.0 ** -53


def gaussian_block(n: int, l: int, seed: int, stream: int = STREAM_X0) -> np.ndarray:
    """n x l matrix of independent N(0, 1) draws (float64), layout as in the module doc."""
    total = n * l
    nblk = (total + 3) // 4
    b = np.arange(nblk, dtype=np.uint64)
    w = philox4x64_10(b, 0, 0, 0, seed, stream)
    z = np.empty((nblk, 4), dtype=np.float64)
    for p in range(2):
        u1 = u24(w[2 * p])
        u2 = u24(w[2 * p + 1])
        r = np.sqrt(-2.0 * np.log(u1))
        z[:, 2 * p] = r * np.cos(2.0 * np.pi * u2)
        z[:, 2 * p + 1] = r * np.sin(2.0 * np.pi * u2)
    flat = z.reshape(-1)[:total]
    return flat.reshape(l, n).T.copy()


def kmeanspp_uniform(seed: int, r: int) -> float:
    """The uniform in [0, 1) that k-means++ round ``r`` (0-based) consumes."""
    w = philox4x64_10(np.uint64(r), 0, 0, 0, seed, STREAM_KMEANSPP)
    return float(u53(w[0]))
