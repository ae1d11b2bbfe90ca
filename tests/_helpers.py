"""Shared helpers for the GPU parity tests (test infrastructure, not product code)."""
import numpy as np

from oracle import spectral


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
