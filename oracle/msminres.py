"""Multi-shift MINRES (App. C, FP64).

One Lanczos process on (K, b) is shared by every shift t_q (the observation
before Eq. minres_qr_shifted: the Lanczos factorisation of K + tI is that of K
with T_J + tI).  Each shift then runs its own MINRES on T_J + t_q I
(Eq. minres_qr_shifted): its own Givens QR, its own step phi and its own
search directions d (App. C.2 prose).  The printed Givens lines of the
algorithms do not reproduce MINRES as written (the updated eta is eta^2/rho,
||b|| scales twice), so the standard Paige-Saunders recurrence that Eq.
minres_qr_shifted defines is used, for each shift with alpha_bar = alpha_j + t:

  initial: c_0 = c_{-1} = 1, s_0 = s_{-1} = 0, phibar = beta_1, d_0 = d_{-1} = 0, x = 0
  step j:
    eps     = s_{j-2} beta_j          ; deltabar = c_{j-2} beta_j
    delta   = c_{j-1} deltabar + s_{j-1} alpha_bar
    gammabar = -s_{j-1} deltabar + c_{j-1} alpha_bar
    gamma   = sqrt(gammabar^2 + beta_{j+1}^2)
    c_j = gammabar / gamma ;  s_j = beta_{j+1} / gamma
    tau = c_j phibar ;  phibar <- -s_j phibar     (|phibar| = residual norm)
    d_j = (q_j - delta d_{j-1} - eps d_{j-2}) / gamma
    x_j = x_{j-1} + tau d_j

(beta_j at j = 1 multiplies d_0 = d_{-1} = 0 and is taken as 0.)

Columns of a block of right-hand sides are independent problems that share
the block MVM; each column has its own Lanczos scalars and stops on its own.
"""
from __future__ import annotations

import numpy as np

BREAKDOWN_RTOL = 1e-13


def msminres(mvm, B: np.ndarray, shifts: np.ndarray, max_iter: int, stop=None):
    """Solve (K + t_q I) x = b for every shift and every column of ``B``.

    ``B``: (n, T).  ``stop(j, phibar, X, alphas, betas) -> bool[T]`` is
    called after each step with the per-shift residual estimates ``phibar``
    (Q, T), the current solutions ``X`` (Q, n, T) and each column's Lanczos
    coefficients so far (lists as in the returned info); columns for which it
    returns True freeze.  Returns (X, info) with info holding the iteration count per
    column, |phibar|, and the Lanczos coefficients per column.
    """
    B = np.asarray(B, dtype=np.float64)
    shifts = np.asarray(shifts, dtype=np.float64)
    n, T = B.shape
    Q = shifts.shape[0]
    beta1 = np.linalg.norm(B, axis=0)                      # (T,)
    active = beta1 > 0.0
    safe = np.where(active, beta1, 1.0)
    q_prev = np.zeros_like(B)
    q = B / safe
    beta_j = np.zeros(T)                                    # beta_j (0 at j = 1)
    c1 = np.ones((Q, T)); s1 = np.zeros((Q, T))             # c_{j-1}, s_{j-1}
    c2 = np.ones((Q, T)); s2 = np.zeros((Q, T))             # c_{j-2}, s_{j-2}
    phibar = np.tile(beta1, (Q, 1))
    d1 = np.zeros((Q, n, T)); d2 = np.zeros((Q, n, T))      # d_{j-1}, d_{j-2}
    X = np.zeros((Q, n, T))
    iters = np.zeros(T, dtype=np.int64)
    alphas = [[] for _ in range(T)]
    betas = [[b] for b in beta1]
    for j in range(1, max_iter + 1):
        if not active.any():
            break
        # Lanczos step (shared by all shifts).
        p = mvm(q) - beta_j * q_prev
        alpha = np.einsum("ic,ic->c", q, p)
        p = p - alpha * q
        beta_next = np.linalg.norm(p, axis=0)
        breakdown = beta_next <= BREAKDOWN_RTOL * (np.abs(alpha) + beta_j)
        beta_next = np.where(breakdown, 0.0, beta_next)
        # Per-shift Givens QR update of T_j + t_q I.
        abar = alpha[None, :] + shifts[:, None]
        eps = s2 * beta_j
        deltabar = c2 * beta_j
        delta = c1 * deltabar + s1 * abar
        gammabar = -s1 * deltabar + c1 * abar
        gamma = np.sqrt(gammabar ** 2 + beta_next[None, :] ** 2)
        cj = gammabar / gamma
        sj = beta_next[None, :] / gamma
        tau = cj * phibar
        phibar_new = -sj * phibar
        # Per-shift direction and solution updates.
        d_new = (q[None] - delta[:, None, :] * d1 - eps[:, None, :] * d2) / gamma[:, None, :]
        X_new = X + tau[:, None, :] * d_new
        # Commit only for active columns.
        m = active
        X[:, :, m] = X_new[:, :, m]
        d2[:, :, m] = d1[:, :, m]; d1[:, :, m] = d_new[:, :, m]
        c2[:, m] = c1[:, m]; s2[:, m] = s1[:, m]
        c1[:, m] = cj[:, m]; s1[:, m] = sj[:, m]
        phibar[:, m] = phibar_new[:, m]
        iters[m] = j
        for c in np.nonzero(m)[0]:
            alphas[c].append(alpha[c]); betas[c].append(beta_next[c])
        q_next = np.where(breakdown, 0.0, p / np.where(beta_next > 0, beta_next, 1.0))
        q_prev = np.where(m, q, q_prev)
        q = np.where(m, q_next, q)
        beta_j = np.where(m, beta_next, beta_j)
        done = breakdown.copy()
        if stop is not None:
            done |= stop(j, phibar, X, alphas, betas)
        active = active & ~done
    info = dict(iters=iters, phibar=phibar, alpha=[np.array(a) for a in alphas],
                beta=[np.array(b) for b in betas], beta1=beta1)
    return X, info
