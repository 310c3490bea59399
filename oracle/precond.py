"""Preconditioned msMINRES-CIQ (Sec. 3 "Preconditioning"; App. "Preconditioning
msMINRES-CIQ", Eq. not_a_sqrt, Eq. precond_sqrt, Eq. precond_sqrt_inverse), FP64.

TEST INFRASTRUCTURE: only tests/, the smoke check and the bench's CPU legs use it.

With a symmetric positive definite preconditioner P ~ K, msMINRES run on the
preconditioned operator A = P^{-1/2} K P^{-1/2} gives the shifted solves

    P^{-1/2} (A + t_q I)^{-1} P^{-1/2} = (K + t_q P)^{-1},

and the quadrature of Eq. contour_integral_quad applied to the start vector
z = P^{1/2} b yields (Eq. precond_sqrt_inverse, Eq. precond_sqrt)

    R' b = sum_q w_q (K + t_q P)^{-1} z  ~  P^{-1/2} A^{-1/2} b,   R' R'^T = K^{-1},
    R  b = K R' b                          ~  K P^{-1/2} A^{-1/2} b, R  R^T  = K,

roots of K^{-1} and K that equal K^{-1/2}, K^{1/2} up to an orthogonal
rotation; the nodes (w_q, t_q) cover the spectrum of A (the spectrum of P^{-1}K).

Preconditioner (App. "Preconditioning msMINRES-CIQ", last paragraph): the
partial pivoted Cholesky factor Lbar of K_XX (rank R, Harbrecht, Peters and
Schneider 2012), P = Lbar Lbar^T + sigma^2 I.  Readings where the paper is
silent:

  * pivoted Cholesky: greedy, the pivot is the largest remaining diagonal
    entry of K_XX - L L^T (the first index on ties); it runs on K_XX, the
    kernel without the noise term (P adds sigma^2 I back);
  * P^{-1} by the matrix inversion lemma (the paper's "solves using the
    matrix inversion lemma"): P^{-1} v = (v - L (sigma^2 I + L^T L)^{-1} L^T v) / sigma^2;
  * P^{1/2} b: P is low rank plus a multiple of I, so its principal root has
    a closed form from the R x R eigendecomposition L^T L = U diag(s) U^T:
    P^{1/2} = sigma I + L U diag(1 / (sqrt(s + sigma^2) + sigma)) U^T L^T
    (the paper runs CIQ on P only when P does not decompose readily);
  * bounds: K_XX - L L^T is a Schur complement, so P <= K and every
    eigenvalue of P^{-1}K is >= 1: lambda_min = 1 (the analogue of the sigma^2
    reading without a preconditioner), lambda_max = 1.05 theta_max of a
    preconditioned Lanczos pre-pass;
  * K^{1/2}: the identity form K (K + tP)^{-1} = I - t P (K + tP)^{-1}, i.e.
    R b = (sum w) z - P sum_q w_q t_q x_q (no extra kernel MVM), or
    sqrt_form="mvm": Eq. precond_sqrt as printed, R b = K (R' b), where R' b
    is solved and stopped exactly as for op="invsqrt" (the identity form's
    error in the space of K can exceed the bound its stop rule uses by up to
    sqrt(kappa(P)); the printed form's does not, at one more kernel MVM);
  * stopping: the rules of the unpreconditioned solve evaluated in the space
    msMINRES works in (that of A): |phibar_q| there is the P^{-1}-norm of the
    residual of (K + t_q P) x = z, the estimate's norm is its A-space norm
    (||R'b||_P, ||R b||_{P^{-1}}), and the scalar norms of the stored-basis
    rule are ||b|| sqrt(alpha_1) = ||A^{1/2} b|| and the Gauss rule of T_j.
"""
from __future__ import annotations

import numpy as np

from .ciq import gauss_invsqrt_norm
from .lanczos import ritz_extremes
from .quadrature import quad_nodes

BREAKDOWN_RTOL = 1e-13


# ----------------------------------------------------------- preconditioner --
def pivoted_cholesky(diag, column, rank):
    """Partial pivoted Cholesky of an SPD matrix known by its diagonal and columns.

    ``diag``: the n diagonal entries; ``column(i)``: column i (n entries).
    Greedy pivoting on the largest remaining diagonal entry.  Returns
    (L, piv): L is n x r (r <= rank; fewer when the remaining diagonal is all
    zero), piv the pivots in order.  K - L L^T is the Schur complement of the
    pivot block: positive semidefinite, zero in the pivot rows and columns.
    """
    d = np.array(diag, dtype=np.float64)
    n = d.shape[0]
    rank = min(rank, n)
    L = np.zeros((n, rank))
    piv = []
    for k in range(rank):
        i = int(np.argmax(d))
        if d[i] <= 0.0:
            L = L[:, :k]
            break
        col = np.asarray(column(i), dtype=np.float64) - L[:, :k] @ L[i, :k]
        col[piv] = 0.0                        # earlier pivot rows of the Schur complement are exactly 0
        piv.append(i)
        L[:, k] = col / np.sqrt(d[i])
        d = d - L[:, k] ** 2
        d[piv] = 0.0                          # and so is the diagonal at every pivot
    return L, np.array(piv, dtype=np.int64)


class Preconditioner:
    """P = L L^T + sigma^2 I with its inverse (Woodbury) and principal root."""

    def __init__(self, L: np.ndarray, noise: float):
        self.L = np.asarray(L, dtype=np.float64)
        self.noise = float(noise)
        r = self.L.shape[1]
        self.C = self.noise * np.eye(r) + self.L.T @ self.L          # sigma^2 I + L^T L
        s, U = np.linalg.eigh(self.L.T @ self.L)
        self.gram_eig = np.clip(s, 0.0, None)
        self.U = U

    def matvec(self, V):
        """P V."""
        V = np.asarray(V, dtype=np.float64)
        return self.noise * V + self.L @ (self.L.T @ V)

    def solve(self, V):
        """P^{-1} V by the matrix inversion lemma."""
        V = np.asarray(V, dtype=np.float64)
        return (V - self.L @ np.linalg.solve(self.C, self.L.T @ V)) / self.noise

    def sqrt(self, V):
        """P^{1/2} V (closed form, see module docstring)."""
        V = np.asarray(V, dtype=np.float64)
        sig = np.sqrt(self.noise)
        g = 1.0 / (np.sqrt(self.gram_eig + self.noise) + sig)
        coef = self.U.T @ (self.L.T @ V)
        coef = coef * (g[:, None] if coef.ndim == 2 else g)
        return sig * V + self.L @ (self.U @ coef)

    def dense(self):
        return self.L @ self.L.T + self.noise * np.eye(self.L.shape[0])


def kernel_preconditioner(K_XX_diag, K_XX_column, noise, rank):
    L, piv = pivoted_cholesky(K_XX_diag, K_XX_column, rank)
    return Preconditioner(L, noise), piv


# ------------------------------------------------ preconditioned Lanczos ----
def precond_lanczos(mvm, psolve, z, J):
    """J steps of Lanczos on A = P^{-1/2} K P^{-1/2} from P^{-1/2} z, in the
    coordinates of K (Paige and Saunders 1975; Choi 2006, Ch. 3.4).

    With u_j = P^{-1/2} v_j and w_j = P^{1/2} v_j for the Lanczos vectors v_j
    of A:  beta_1 = sqrt(z^T P^{-1} z), w_1 = z / beta_1, u_1 = P^{-1} z / beta_1;
      p = K u_j - beta_j w_{j-1};  alpha_j = u_j^T p;  p -= alpha_j w_j;
      beta_{j+1} = sqrt(p^T P^{-1} p);  w_{j+1} = p / beta_{j+1};
      u_{j+1} = P^{-1} p / beta_{j+1}.
    Returns (alpha, beta) as lanczos.lanczos does (beta[0] = beta_1).
    """
    z = np.asarray(z, dtype=np.float64)
    y = psolve(z)
    beta1 = float(np.sqrt(z @ y))
    alphas, betas = [], [beta1]
    w_prev = np.zeros_like(z)
    w, u = z / beta1, y / beta1
    for _ in range(J):
        p = mvm(u) - betas[-1] * w_prev if alphas else mvm(u)
        a = float(u @ p)
        p = p - a * w
        y = psolve(p)
        b = float(np.sqrt(max(p @ y, 0.0)))
        alphas.append(a)
        betas.append(b)
        if b == 0.0:
            break
        w_prev, w, u = w, p / b, y / b
    return np.array(alphas), np.array(betas)


def precond_msminres(mvm, psolve, Z, shifts, max_iter, stop=None):
    """(K + t_q P) x = z for every shift and every column of Z (n, T).

    The multi-shift MINRES of App. C (Paige-Saunders recurrence, one Givens
    QR per shift, oracle/msminres.py) on the preconditioned Lanczos process
    above: the shift enters as alpha_j + t_q because A + tI has the Lanczos
    tridiagonal T_j + tI, and the search directions live in the u coordinates,
    so the iterates x_q are the solutions of the original shifted systems.
    |phibar_q| is the P^{-1}-norm of the residual z - (K + t_q P) x_q.
    ``stop(j, phibar, X, alphas, betas)`` as in oracle/msminres.py.
    """
    Z = np.asarray(Z, dtype=np.float64)
    shifts = np.asarray(shifts, dtype=np.float64)
    n, T = Z.shape
    Q = shifts.shape[0]
    Y = psolve(Z)
    beta1 = np.sqrt(np.maximum(np.einsum("ic,ic->c", Z, Y), 0.0))
    active = beta1 > 0.0
    safe = np.where(active, beta1, 1.0)
    w_prev = np.zeros_like(Z)
    w, u = Z / safe, Y / safe
    beta_j = np.zeros(T)
    c1 = np.ones((Q, T)); s1 = np.zeros((Q, T))
    c2 = np.ones((Q, T)); s2 = np.zeros((Q, T))
    phibar = np.tile(beta1, (Q, 1))
    d1 = np.zeros((Q, n, T)); d2 = np.zeros((Q, n, T))
    X = np.zeros((Q, n, T))
    iters = np.zeros(T, dtype=np.int64)
    alphas = [[] for _ in range(T)]
    betas = [[b] for b in beta1]
    for j in range(1, max_iter + 1):
        if not active.any():
            break
        # Preconditioned Lanczos step (shared by all shifts).
        p = mvm(u) - beta_j * w_prev
        alpha = np.einsum("ic,ic->c", u, p)
        p = p - alpha * w
        y = psolve(p)
        beta_next = np.sqrt(np.maximum(np.einsum("ic,ic->c", p, y), 0.0))
        breakdown = beta_next <= BREAKDOWN_RTOL * (np.abs(alpha) + beta_j)
        beta_next = np.where(breakdown, 0.0, beta_next)
        # Per-shift Givens QR update of T_j + t_q I (as oracle/msminres.py).
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
        d_new = (u[None] - delta[:, None, :] * d1 - eps[:, None, :] * d2) / gamma[:, None, :]
        X_new = X + tau[:, None, :] * d_new
        m = active
        X[:, :, m] = X_new[:, :, m]
        d2[:, :, m] = d1[:, :, m]; d1[:, :, m] = d_new[:, :, m]
        c2[:, m] = c1[:, m]; s2[:, m] = s1[:, m]
        c1[:, m] = cj[:, m]; s1[:, m] = sj[:, m]
        phibar[:, m] = phibar_new[:, m]
        iters[m] = j
        for c in np.nonzero(m)[0]:
            alphas[c].append(alpha[c]); betas[c].append(beta_next[c])
        safe_b = np.where(beta_next > 0, beta_next, 1.0)
        w_next = np.where(breakdown, 0.0, p / safe_b)
        u_next = np.where(breakdown, 0.0, y / safe_b)
        w_prev = np.where(m, w, w_prev)
        w = np.where(m, w_next, w)
        u = np.where(m, u_next, u)
        beta_j = np.where(m, beta_next, beta_j)
        done = breakdown.copy()
        if stop is not None:
            done |= stop(j, phibar, X, alphas, betas)
        active = active & ~done
    info = dict(iters=iters, phibar=phibar, alpha=[np.array(a) for a in alphas],
                beta=[np.array(b) for b in betas], beta1=beta1)
    return X, info


# ------------------------------------------------------------ CIQ on top ----
def precond_bounds(mvm, pre: Preconditioner, start, iters, lmax_margin=1.05):
    """lambda_min = 1 (P <= K), lambda_max = lmax_margin theta_max of a
    preconditioned Lanczos pre-pass of ``iters`` steps from P^{1/2} start."""
    a, b = precond_lanczos(mvm, pre.solve, pre.sqrt(start), iters)
    th_min, th_max = ritz_extremes(a, b)
    return dict(ritz_min=th_min, ritz_max=th_max, lmin=1.0, lmax=lmax_margin * th_max)


def ciq_precond_apply(mvm, pre: Preconditioner, B, Q, op, tol=0.0, max_iter=200, stop_rule="residual",
                      start=None, lanczos_iters=10, lmin=None, lmax=None, nodes=None, sqrt_form="identity",
                      lmax_margin=1.05, errbound_norm="estimate"):
    """R B (op="sqrt", Eq. precond_sqrt) or R' B (op="invsqrt",
    Eq. precond_sqrt_inverse) for B of shape (T, n); returns (A, info), A (T, n).

    Steps: z = P^{1/2} b; nodes over the spectrum of P^{-1}K; multi-shift
    MINRES for (K + t_q P) x_q = z; R' b = sum_q w_q x_q and
    R b = (sum w) z - P sum_q w_q t_q x_q (or K sum_q w_q x_q).
    """
    B = np.asarray(B, dtype=np.float64)
    Bc = B.T
    Z = pre.sqrt(Bc)
    info = {}
    if nodes is not None:
        w, t = (np.asarray(v, dtype=np.float64) for v in nodes)
        info.update(lmin=lmin, lmax=lmax)
    else:
        if lmin is None or lmax is None:
            if start is None:
                raise ValueError("need a Lanczos start vector, explicit bounds or nodes")
            bnd = precond_bounds(mvm, pre, start, lanczos_iters, lmax_margin)
            info.update(bnd)
            lmin, lmax = bnd["lmin"], bnd["lmax"]
        else:
            info.update(lmin=lmin, lmax=lmax)
        w, t = quad_nodes(lmin, lmax, Q)
    info.update(w=w, t=t)
    literal = op == "sqrt" and sqrt_form == "mvm"
    solve_op = "invsqrt" if literal else op           # R b = K (R' b): R' b's solve and rule
    coef = w if solve_op == "invsqrt" else w * t
    lmin_b = info.get("lmin") or 0.0

    def estimate(Xs):
        if solve_op == "invsqrt":
            return np.einsum("q,qic->ic", w, Xs)
        return w.sum() * Z - pre.matvec(np.einsum("q,qic->ic", w * t, Xs))

    def a_norm(E):
        # Norm in the space of A: R'b = P^{-1/2} a_A, R b = P^{1/2} a_A.
        M = pre.matvec(E) if solve_op == "invsqrt" else pre.solve(E)
        return np.sqrt(np.maximum(np.einsum("ic,ic->c", E, M), 0.0))

    sqrt_norm = None
    if errbound_norm == "scalar" and solve_op == "sqrt":
        # ||A^{1/2} b|| = sqrt(b^T A b) with P^{-1/2} b = P^{-1} z (one extra MVM
        # here; the device has it as ||b|| sqrt(alpha_1)).
        Y = pre.solve(Z)
        sqrt_norm = np.sqrt(np.maximum(np.einsum("ic,ic->c", Y, mvm(Y)), 0.0))

    def stop(j, phibar, Xs, alphas, betas):
        if tol <= 0.0:
            return np.zeros(phibar.shape[1], dtype=bool)
        if stop_rule == "residual":
            beta1 = np.linalg.norm(Bc, axis=0)
            return np.max(np.abs(phibar), axis=0) <= tol * beta1
        bound = np.sum(coef[:, None] * np.abs(phibar) / (t[:, None] + lmin_b), axis=0)
        if errbound_norm == "scalar":
            den = sqrt_norm if solve_op == "sqrt" else np.array(
                [gauss_invsqrt_norm(a, b) for a, b in zip(alphas, betas)])
            return bound <= tol * (1.0 - 2.0 * tol) * den
        return bound <= tol * a_norm(estimate(Xs))

    Xs, minfo = precond_msminres(mvm, pre.solve, Z, t, max_iter, stop)
    info.update(minfo)
    A = estimate(Xs)
    if literal:
        A = mvm(A)
    info["errbound"] = np.sum(coef[:, None] * np.abs(minfo["phibar"]) / (t[:, None] + lmin_b), axis=0)
    return A.T, info


# ------------------------------------------------- exact rotated roots (O1) --
def rotated_roots_exact(K, P, B):
    """R B and R' B by dense eigendecompositions (FP64), B of shape (T, n).

    P^{+-1/2} from eigh(P); A = P^{-1/2} K P^{-1/2} and A^{-1/2} from eigh(A);
    R b = K P^{-1/2} A^{-1/2} b and R' b = P^{-1/2} A^{-1/2} b, with b itself
    as A's argument since P^{-1/2} (P^{1/2} b) = b (Eq. precond_sqrt,
    Eq. precond_sqrt_inverse).
    """
    from .eig import eigh

    K = np.asarray(K, dtype=np.float64)
    P = np.asarray(P, dtype=np.float64)
    lp, Vp = eigh(P)
    P_mhalf = (Vp * lp ** -0.5) @ Vp.T
    A = P_mhalf @ K @ P_mhalf
    A = 0.5 * (A + A.T)
    la, Va = eigh(A)
    Bc = np.asarray(B, dtype=np.float64).T
    core = Va @ ((Va.T @ Bc) * (la ** -0.5)[:, None])
    inv = P_mhalf @ core
    return (K @ inv).T, inv.T
