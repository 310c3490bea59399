"""Kernel functions and kernel matrix-vector products (FP64).

The paper names the RBF and Matern-5/2 kernels (Sec. 4, Sec. 5, App. E-F) but
never writes them out.  Reading used throughout, isotropic lengthscale ``l``,
outputscale ``s`` multiplying the kernel, ``r = ||x - x'||``:

    RBF          k(r) = s * exp(-r^2 / (2 l^2))
    Matern-5/2   k(r) = s * (1 + sqrt(5) r / l + 5 r^2 / (3 l^2)) * exp(-sqrt(5) r / l)

and the matrix whose square root is taken is K = K_XX + sigma^2 I
(Sec. 3, "K = K_XX + sigma^2 I" in the problem statement of msMINRES-CIQ).

Distances are formed from coordinate differences (no norm expansion), which
is the plain definition.
"""
from __future__ import annotations

import numpy as np

SQRT5 = np.sqrt(5.0)


def kernel_of_r2(r2: np.ndarray, kind: str, lengthscale: float, outputscale: float) -> np.ndarray:
    """k as a function of the squared distance ``r2`` (see module docstring)."""
    if kind == "rbf":
        return outputscale * np.exp(-0.5 * r2 / lengthscale ** 2)
    if kind == "matern52":
        rl = np.sqrt(r2) / lengthscale
        return outputscale * (1.0 + SQRT5 * rl + (5.0 / 3.0) * rl * rl) * np.exp(-SQRT5 * rl)
    raise ValueError(f"unknown kernel {kind!r}")


def sqdist(X1: np.ndarray, X2: np.ndarray) -> np.ndarray:
    """Squared Euclidean distances from coordinate differences, shape (n1, n2)."""
    X1 = np.asarray(X1, dtype=np.float64)
    X2 = np.asarray(X2, dtype=np.float64)
    r2 = np.zeros((X1.shape[0], X2.shape[0]))
    for k in range(X1.shape[1]):
        diff = X1[:, k][:, None] - X2[:, k][None, :]
        r2 += diff * diff
    return r2


def kernel_matrix(X1, X2, kind, lengthscale, outputscale) -> np.ndarray:
    """K_{X1 X2} (no noise term)."""
    return kernel_of_r2(sqdist(X1, X2), kind, lengthscale, outputscale)


def dense_K(X, kind, lengthscale, outputscale, noise) -> np.ndarray:
    """K = K_XX + sigma^2 I as a dense FP64 matrix."""
    K = kernel_matrix(X, X, kind, lengthscale, outputscale)
    K[np.diag_indices_from(K)] += noise
    return K


def mvm(X, kind, lengthscale, outputscale, noise, V, rows_per_block: int = 2048) -> np.ndarray:
    """(K_XX + sigma^2 I) V without storing K.

    ``V`` has shape (n, t) (columns are vectors) or (n,).  Row blocks of K are
    formed one at a time only to bound memory; every output entry is the plain
    dot product of one row of K with V.
    """
    V = np.asarray(V, dtype=np.float64)
    out = np.empty_like(V)
    n = X.shape[0]
    for r0 in range(0, n, rows_per_block):
        r1 = min(n, r0 + rows_per_block)
        Kb = kernel_matrix(X[r0:r1], X, kind, lengthscale, outputscale)
        out[r0:r1] = Kb @ V
    out += noise * V
    return out
