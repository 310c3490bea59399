"""O2: plain serial msMINRES-CIQ (Algorithm "ciq"; Eq. contour_integral_quad).

  1. nodes: Lanczos extreme eigenvalues -> (lambda_min, lambda_max) -> (w_q, t_q)
     (Algorithm "quadrature", App. B);
  2. msMINRES for (t_q I + K)^{-1} b, q = 1..Q, sharing one Lanczos process (App. C);
  3. K^{-1/2} b ~= sum_q w_q (t_q I + K)^{-1} b.

K^{1/2} b: Eq. contour_integral_quad writes K sum_q w_q (t_q I + K)^{-1} b.
Since K (t I + K)^{-1} = I - t (t I + K)^{-1}, the same quantity is
(sum_q w_q) b - sum_q w_q t_q (t_q I + K)^{-1} b, which needs no extra MVM.
That identity form is the default reading; ``sqrt_form="mvm"`` applies K
literally.

Stopping rules (the paper's "relative residual" is not defined further):
  "residual":  max_q |phibar_q| / ||b|| <= tol            (per column)
  "errbound":  sum_q c_q |phibar_q| / (t_q + lambda_min) <= tol ||a_j||
               with c_q = w_q (K^{-1/2}) or w_q t_q (K^{1/2}), because
               ||x_q - x_q*|| <= ||r_q|| / lambda_min(K + t_q I).
Both are evaluated after the update of step j, on a_j, the estimate at step j.

``errbound_norm="scalar"`` replaces ||a_j|| by a norm that needs no vector:
  K^{1/2}:  ||K^{1/2} b|| = sqrt(b^T K b)  (one extra MVM here; a Lanczos
            implementation has it as ||b|| sqrt(alpha_1));
  K^{-1/2}: sqrt(||b||^2 e_1^T T_j^{-1} e_1) <= ||K^{-1/2} b||, the Gauss
            quadrature rule of the Lanczos tridiagonal T_j (from below);
both times (1 - 2 tol), so that the bound is <= tol ||a_j|| at the stop as
well (||a_j|| >= ||a*|| - bound).
"""
from __future__ import annotations

import numpy as np
import scipy.linalg

from . import kernels
from .lanczos import lanczos, ritz_extremes, spectral_bounds
from .msminres import msminres
from .quadrature import quad_nodes


def make_mvm(X, kind, lengthscale, outputscale, noise):
    X = np.asarray(X, dtype=np.float64)

    def mvm(V):
        return kernels.mvm(X, kind, lengthscale, outputscale, noise, V)
    return mvm


def lanczos_bounds(mvm, start, iters, noise, lmax_margin=1.05, lmin_div=100.0):
    """Algorithm "quadrature", first two lines, plus the margin reading."""
    alpha, beta = lanczos(mvm, start, iters)
    th_min, th_max = ritz_extremes(alpha, beta)
    lmin, lmax = spectral_bounds(th_min, th_max, noise, lmax_margin, lmin_div)
    return dict(ritz_min=th_min, ritz_max=th_max, lmin=lmin, lmax=lmax, alpha=alpha, beta=beta)


def gauss_invsqrt_norm(alpha, beta):
    """||b|| sqrt(e_1^T T_j^{-1} e_1), the Gauss quadrature rule for b^T K^{-1} b.

    ``alpha`` (j entries) and ``beta`` (beta[0] = ||b||, then beta_2.. as the
    msMINRES info lists them) give the Lanczos tridiagonal T_j, solved here
    with a banded LAPACK solve.  For SPD K this is a lower bound of ||K^{-1/2} b|| that grows
    with j and is exact once the Krylov space is invariant.
    """
    jn = len(alpha)
    if jn == 0:
        return 0.0
    ab = np.zeros((3, jn))                   # T_j in banded storage (super, main, sub)
    ab[0, 1:] = beta[1:jn]
    ab[1] = alpha
    ab[2, :-1] = beta[1:jn]
    e1 = np.zeros(jn)
    e1[0] = 1.0
    return beta[0] * np.sqrt(max(scipy.linalg.solve_banded((1, 1), ab, e1)[0], 0.0))


def ciq_apply(mvm, B, Q, op, tol=0.0, max_iter=200, stop_rule="residual", noise=0.0,
              start=None, lanczos_iters=10, lmin=None, lmax=None, nodes=None,
              sqrt_form="identity", lmax_margin=1.05, lmin_div=100.0, errbound_norm="estimate"):
    """K^{1/2} B (op="sqrt") or K^{-1/2} B (op="invsqrt") for B of shape (T, n).

    Returns (A, info) with A of shape (T, n).
    """
    B = np.asarray(B, dtype=np.float64)
    Bc = B.T                                            # columns are right-hand sides
    info = {}
    if nodes is not None:
        w, t = (np.asarray(v, dtype=np.float64) for v in nodes)
        info.update(lmin=lmin, lmax=lmax)
    else:
        if lmin is None or lmax is None:
            if start is None:
                raise ValueError("need a Lanczos start vector, explicit bounds or nodes")
            bnd = lanczos_bounds(mvm, start, lanczos_iters, noise, lmax_margin, lmin_div)
            info.update(bnd)
            lmin, lmax = bnd["lmin"], bnd["lmax"]
        else:
            info.update(lmin=lmin, lmax=lmax)
        w, t = quad_nodes(lmin, lmax, Q)
    info.update(w=w, t=t)
    coef = w if op == "invsqrt" else w * t
    lmin_b = info.get("lmin") or 0.0

    def estimate(Xs):
        if op == "invsqrt":
            return np.einsum("q,qic->ic", w, Xs)
        return w.sum() * Bc - np.einsum("q,qic->ic", w * t, Xs)

    sqrt_norm = None
    if errbound_norm == "scalar" and op == "sqrt":
        sqrt_norm = np.sqrt(np.einsum("ic,ic->c", Bc, mvm(Bc)))          # ||K^{1/2} b||

    def gauss_norm(alphas, betas):
        return np.array([gauss_invsqrt_norm(a, b) for a, b in zip(alphas, betas)])

    def stop(j, phibar, Xs, alphas, betas):
        if tol <= 0.0:
            return np.zeros(phibar.shape[1], dtype=bool)
        if stop_rule == "residual":
            beta1 = np.linalg.norm(Bc, axis=0)
            return np.max(np.abs(phibar), axis=0) <= tol * beta1
        bound = np.sum(coef[:, None] * np.abs(phibar) / (t[:, None] + lmin_b), axis=0)
        if op == "sqrt" and sqrt_form == "mvm":
            bound = bound * (info.get("lmax") or 1.0)
        if errbound_norm == "scalar":
            den = sqrt_norm if op == "sqrt" else gauss_norm(alphas, betas)
            return bound <= tol * (1.0 - 2.0 * tol) * den
        return bound <= tol * np.linalg.norm(estimate(Xs), axis=0)

    Xs, minfo = msminres(mvm, Bc, t, max_iter, stop)
    info.update(minfo)
    if op == "sqrt" and sqrt_form == "mvm":
        A = mvm(np.einsum("q,qic->ic", w, Xs))
    else:
        A = estimate(Xs)
    info["errbound"] = np.sum(coef[:, None] * np.abs(minfo["phibar"]) / (t[:, None] + lmin_b), axis=0)
    return A.T, info


def ciq_sqrt(X, kind, lengthscale, outputscale, noise, B, Q, **kw):
    """K^{1/2} B for K = K_XX + sigma^2 I; B is (T, n)."""
    mvm = make_mvm(X, kind, lengthscale, outputscale, noise)
    return ciq_apply(mvm, B, Q, "sqrt", noise=noise, **kw)


def ciq_invsqrt(X, kind, lengthscale, outputscale, noise, B, Q, **kw):
    """K^{-1/2} B for K = K_XX + sigma^2 I; B is (T, n)."""
    mvm = make_mvm(X, kind, lengthscale, outputscale, noise)
    return ciq_apply(mvm, B, Q, "invsqrt", noise=noise, **kw)


def dense_mvm(K):
    """MVM with an explicit dense matrix (small problems and synthetic spectra)."""
    K = np.asarray(K, dtype=np.float64)

    def mvm(V):
        return K @ V
    return mvm
