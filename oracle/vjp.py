"""Backward pass of msMINRES-CIQ (Sec. 3.4, Eq. ciq_deriv), FP64, test infrastructure.

Differentiating each term of the quadrature (Eq. contour_integral_quad) with
the nodes held fixed: for a = sum_q w_q (t_q I + K)^{-1} b ~ K^{-1/2} b and a
loss L with dL/da = g,

    dL/dK = -1/2 sum_q w_q (t_q I + K)^{-1} (g b^T + b g^T) (t_q I + K)^{-1}
          = -1/2 sum_q w_q (y_q x_q^T + x_q y_q^T),

x_q = (t_q I + K)^{-1} b, y_q = (t_q I + K)^{-1} g: one more multi-shift solve,
on g.  For a hyperparameter theta of K (symmetric dK/dtheta):

    dL/dtheta = sum_q c_q y_q^T (dK/dtheta) x_q,   c_q = -w_q        (K^{-1/2} b)

and for K^{1/2} b = (sum w) b - sum_q w_q t_q x_q (identity form, R7), c_q =
+w_q t_q.  dL/db is the same operator applied to g (K^{+-1/2} is symmetric):
sum_q w_q y_q, or (sum w) g - sum_q w_q t_q y_q.

dK/dtheta for K = s k(r; l) + sigma^2 I (kernels.py): dK/dsigma^2 = I,
dK/ds = K_XX / s, and dK/dl = s dk/dl with

    RBF         dk/dl = k r^2 / l^3
    Matern-5/2  dk/dl = (z^2 / (3 l)) (1 + z) exp(-z),  z = sqrt(5) r / l.

Everything here is the plain definition written out: dense matrices, no
blocking.  Only tests/ import this module.
"""
from __future__ import annotations

import numpy as np

from .kernels import SQRT5, kernel_of_r2, sqdist
from .msminres import msminres


def dkernel_dl(r2: np.ndarray, kind: str, lengthscale: float, outputscale: float) -> np.ndarray:
    """d k / d lengthscale as a function of the squared distance (see module docstring)."""
    l = lengthscale
    if kind == "rbf":
        return outputscale * np.exp(-0.5 * r2 / l ** 2) * r2 / l ** 3
    if kind == "matern52":
        z = SQRT5 * np.sqrt(r2) / l
        return outputscale * (z * z / (3.0 * l)) * (1.0 + z) * np.exp(-z)
    raise ValueError(f"unknown kernel {kind!r}")


def dK_dtheta(X, kind, lengthscale, outputscale):
    """Dense (dK/dl, dK/ds, dK/dsigma^2)."""
    r2 = sqdist(X, X)
    dl = dkernel_dl(r2, kind, lengthscale, outputscale)
    ds = kernel_of_r2(r2, kind, lengthscale, 1.0)                 # K_XX / s
    return dl, ds, np.eye(r2.shape[0])


def ciq_vjp(K, dKs, B, G, w, t, op, max_iter):
    """a = CIQ(B), dL/dB and dL/dtheta for L = sum_c g_c . a_c at fixed nodes.

    K: dense SPD matrix; dKs: list of dense dK/dtheta; B, G: (T, n); w, t:
    nodes; op "invsqrt" or "sqrt".  Returns (A, grad_B, grad_theta) with A and
    grad_B of shape (T, n) and grad_theta one entry per matrix in dKs.
    """
    B = np.asarray(B, dtype=np.float64)
    G = np.asarray(G, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    mvm = lambda V: K @ V                                         # noqa: E731
    Xs, _ = msminres(mvm, B.T, t, max_iter)                        # (Q, n, T): x_q per column
    Ys, _ = msminres(mvm, G.T, t, max_iter)                        # y_q
    if op == "invsqrt":
        A = np.einsum("q,qic->ic", w, Xs)
        gB = np.einsum("q,qic->ic", w, Ys)
        c = -w
    else:
        A = w.sum() * B.T - np.einsum("q,qic->ic", w * t, Xs)
        gB = w.sum() * G.T - np.einsum("q,qic->ic", w * t, Ys)
        c = w * t
    grads = []
    for D in dKs:
        DX = np.einsum("ij,qjc->qic", D, Xs)
        grads.append(float(np.einsum("q,qic,qic->", c, Ys, DX)))
    return A.T, gB.T, np.array(grads)
