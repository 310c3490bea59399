"""Lanczos process and extreme-eigenvalue estimates (App. B.2, FP64).

Lanczos (the three-term recurrence described in App. B.2 and used inside
Algorithm "msMINRES"), with the reading adopted for the garbled initial lines
of the printed algorithms:

  beta_1 = ||b||,  q_0 = 0,  q_1 = b / beta_1
  for j = 1..J:
    p         = K q_j - beta_j q_{j-1}
    alpha_j   = q_j^T p
    p         = p - alpha_j q_j
    beta_{j+1} = ||p||
    q_{j+1}   = p / beta_{j+1}

No reorthogonalisation (the paper argues it is not needed for solves).
T_J = tridiag(beta_2..beta_J; alpha_1..alpha_J; beta_2..beta_J).

Bounds (App. B.2 asks for "slightly larger and smaller" values than the Ritz
extremes and gives no margin).  Reading:
  lambda_max_used = 1.05 theta_max(T_J)
  lambda_min_used = sigma^2                  if sigma^2 > 0 (K_XX is PSD, so
                                             lambda_min(K) >= sigma^2 exactly)
                  = theta_min(T_J) / 100     otherwise (a heuristic: pinned
                                             against LAPACK's lambda_min on the
                                             Q-sweep matrices, not a bound).
"""
from __future__ import annotations

import numpy as np


def lanczos(mvm, b: np.ndarray, J: int):
    """Run J Lanczos steps on vector ``b``.

    Returns (alpha[J'], beta[J'+1]) with beta[0] = ||b|| = beta_1 and
    beta[j] = beta_{j+1}; J' <= J is smaller when an invariant subspace is
    reached (beta_{j+1} = 0).
    """
    b = np.asarray(b, dtype=np.float64)
    beta1 = np.linalg.norm(b)
    alphas, betas = [], [beta1]
    q_prev = np.zeros_like(b)
    q = b / beta1
    for _ in range(J):
        p = mvm(q) - betas[-1] * q_prev if alphas else mvm(q)
        alpha = float(q @ p)
        p = p - alpha * q
        beta = float(np.linalg.norm(p))
        alphas.append(alpha)
        betas.append(beta)
        if beta == 0.0:
            break
        q_prev, q = q, p / beta
    return np.array(alphas), np.array(betas)


def tridiagonal(alpha: np.ndarray, beta: np.ndarray) -> np.ndarray:
    """Dense T_J from alpha_1..alpha_J and beta_2..beta_J (``beta[1:J]``)."""
    J = len(alpha)
    T = np.diag(alpha)
    if J > 1:
        off = beta[1:J]
        T += np.diag(off, 1) + np.diag(off, -1)
    return T


def ritz_extremes(alpha: np.ndarray, beta: np.ndarray):
    """(theta_min, theta_max) of T_J via LAPACK's symmetric eigensolver."""
    ev = np.linalg.eigvalsh(tridiagonal(alpha, beta))
    return float(ev[0]), float(ev[-1])


def spectral_bounds(theta_min: float, theta_max: float, noise: float,
                    lmax_margin: float = 1.05, lmin_div: float = 100.0):
    """(lambda_min_used, lambda_max_used) from Ritz extremes (module docstring)."""
    lmax = lmax_margin * theta_max
    lmin = noise if noise > 0.0 else theta_min / lmin_div
    return lmin, lmax
