"""O1: the definition of the principal square root (FP64 LAPACK).

For symmetric positive definite K = V diag(lambda) V^T the principal roots are
K^{1/2} b = V diag(lambda^{1/2}) V^T b and K^{-1/2} b = V diag(lambda^{-1/2}) V^T b.
They are unique (Sec. 2 contrasts this with the Cholesky factor, which is one
of many square roots up to rotation).  msMINRES-CIQ approximates exactly this.
"""
from __future__ import annotations

import numpy as np


def matrix_power_apply(K: np.ndarray, B: np.ndarray, power: float) -> np.ndarray:
    """K^power B for SPD K via ``numpy.linalg.eigh``; ``B`` is (n, T) or (n,)."""
    lam, V = np.linalg.eigh(np.asarray(K, dtype=np.float64))
    if lam[0] <= 0.0:
        raise ValueError("matrix is not positive definite")
    B = np.asarray(B, dtype=np.float64)
    coef = V.T @ B
    scale = lam ** power
    coef = coef * (scale[:, None] if coef.ndim == 2 else scale)
    return V @ coef


def sqrt_apply(K, B):
    """K^{1/2} B."""
    return matrix_power_apply(K, B, 0.5)


def invsqrt_apply(K, B):
    """K^{-1/2} B."""
    return matrix_power_apply(K, B, -0.5)
