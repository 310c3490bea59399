"""Posterior Thompson draws (Sec. 5 "Posterior Sampling for Bayesian
Optimization", Eq. thompson_sample), FP64.

TEST INFRASTRUCTURE: only tests/, the smoke check and the bench's CPU legs use it.

A draw at the candidate set X* (N* points) given training data (X, y) is

    f* = mu*(X*) + COV*(X*)^{1/2} eps,   eps ~ N(0, I),

with the Gaussian-process posterior mean and covariance

    mu*  = m + K*X (K_XX + sigma^2 I)^{-1} (y - m),
    COV* = K** - K*X (K_XX + sigma^2 I)^{-1} K_X* + jitter I.

Readings where the paper is brief: the kernel is Matern-5/2 (or RBF) with
ARD lengthscales, i.e. the isotropic kernel of oracle/kernels.py applied to
the coordinates divided by their own lengthscales (App. BO setup names
"Matern-5/2 with ARD"); the mean is a constant m ("constant mean function");
the 1e-4 the paper adds "to the diagonal of the kernel matrix" is the jitter
of COV*; COV*^{1/2} is the principal root (what msMINRES-CIQ approximates;
Cholesky would give a rotated one, Sec. 2).  With a preconditioner (App.
"Preconditioning msMINRES-CIQ"), the draw uses the rotated root R with
R R^T = COV* that the preconditioned solve defines; any root of COV* gives
draws of the same distribution.
"""
from __future__ import annotations

import numpy as np

from . import eig, kernels


def ard_scale(X, lengthscales):
    """Coordinates divided by their lengthscales (ARD)."""
    X = np.asarray(X, dtype=np.float64)
    return X / np.asarray(lengthscales, dtype=np.float64)[None, :]


def kernel_ard(X1, X2, kind, lengthscales, outputscale):
    """k(x, x') with per-dimension lengthscales (isotropic kernel on scaled points)."""
    return kernels.kernel_matrix(ard_scale(X1, lengthscales), ard_scale(X2, lengthscales), kind, 1.0, outputscale)


def posterior(Xtr, y, Xc, kind, lengthscales, outputscale, noise, jitter, mean):
    """(mu*, COV*) dense, from the formulas in the module docstring."""
    Xtr = np.asarray(Xtr, dtype=np.float64).reshape(-1, np.asarray(Xc).shape[1])
    Kcc = kernel_ard(Xc, Xc, kind, lengthscales, outputscale)
    nc = Kcc.shape[0]
    if Xtr.shape[0] == 0:
        return np.full(nc, float(mean)), Kcc + jitter * np.eye(nc)
    M = kernel_ard(Xtr, Xtr, kind, lengthscales, outputscale) + noise * np.eye(Xtr.shape[0])
    Kcx = kernel_ard(Xc, Xtr, kind, lengthscales, outputscale)
    mu = mean + Kcx @ np.linalg.solve(M, np.asarray(y, dtype=np.float64) - mean)
    cov = Kcc - Kcx @ np.linalg.solve(M, Kcx.T) + jitter * np.eye(nc)
    return mu, 0.5 * (cov + cov.T)


def thompson_draws(mu, cov, eps):
    """O1: mu + COV^{1/2} eps for eps of shape (T, N*) (rows are draws)."""
    return mu[None, :] + eig.sqrt_apply(cov, np.asarray(eps, dtype=np.float64).T).T


def preconditioned_draws(mu, cov, jitter, rank, eps):
    """mu + R eps for eps of shape (T, N*): R = P^{1/2} A^{1/2}, A = P^{-1/2}
    COV* P^{-1/2}, P = L L^T + jitter I with L the rank-`rank` pivoted Cholesky
    factor of COV* - jitter I (the noise-free posterior covariance), so that
    R R^T = COV* (Eq. precond_sqrt with sigma^2 = jitter)."""
    from . import precond as PC

    cov = np.asarray(cov, dtype=np.float64)
    n = cov.shape[0]
    C0 = cov - jitter * np.eye(n)
    L, _ = PC.pivoted_cholesky(np.diag(C0).copy(), lambda i: C0[:, i], rank)
    Pm = L @ L.T + jitter * np.eye(n)
    Rb, _ = PC.rotated_roots_exact(cov, Pm, np.asarray(eps, dtype=np.float64))
    return mu[None, :] + Rb
