"""Cyclic Jacobi eigenvalue method for small dense symmetric matrices.

Textbook method (Golub & Van Loan, "Matrix Computations", cyclic Jacobi):
sweep over all off-diagonal pairs (p, q), annihilate a_pq with a plane
rotation chosen by the smaller-angle formula, accumulate the rotations, and
stop when the off-diagonal Frobenius norm falls below ``tol`` times the norm of
the matrix.  Used for n <= a few hundred to get the full spectrum of M.
"""
from __future__ import annotations

import numpy as np


def jacobi_eigh(S: np.ndarray, tol: float = 1e-14, max_sweeps: int = 60):
    """Eigenvalues (ascending) and orthonormal eigenvectors (columns) of symmetric S."""
    A = np.array(S, dtype=np.float64, copy=True)
    n = A.shape[0]
    if not np.allclose(A, A.T, rtol=0, atol=1e-12 * max(1.0, np.abs(A).max())):
        raise ValueError("matrix is not symmetric")
    V = np.eye(n)
    scale = np.linalg.norm(A)
    for _ in range(max_sweeps):
        off = np.linalg.norm(A - np.diag(np.diag(A)))
        if off <= tol * max(scale, 1e-300):
            break
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = A[p, q]
                if apq == 0.0:
                    continue
                theta = (A[q, q] - A[p, p]) / (2.0 * apq)
                t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + np.sqrt(1.0 + theta * theta))
                c = 1.0 / np.sqrt(1.0 + t * t)
                s = t * c
                # A <- J^T A J with J the rotation in the (p, q) plane
                ap = A[:, p].copy()
                aq = A[:, q].copy()
                A[:, p] = c * ap - s * aq
                A[:, q] = s * ap + c * aq
                ap = A[p, :].copy()
                aq = A[q, :].copy()
                A[p, :] = c * ap - s * aq
                A[q, :] = s * ap + c * aq
                A[p, q] = 0.0
                A[q, p] = 0.0
                vp = V[:, p].copy()
                vq = V[:, q].copy()
                V[:, p] = c * vp - s * vq
                V[:, q] = s * vp + c * vq
    else:
        raise RuntimeError("Jacobi did not converge")
    evals = np.diag(A).copy()
    order = np.argsort(evals, kind="stable")
    return evals[order], V[:, order]
