"""Hale-Higham-Trefethen quadrature for K^{-1/2} (App. B, FP64).

Follows Eq. quad_points_and_locations, the sign flip of
Eq. contour_integral_quad_4 and Algorithm "quadrature" in the paper's order:

  k^2 = lambda_min / lambda_max,  k'^2 = 1 - k^2          (the printed
        ``k'^2 <- sqrt(1 - k^2)`` contradicts the definition k' = sqrt(1 - k^2)
        stated with the equation; the definition is used)
  K'  = K(k')                                             (complete integral)
  for q = 1..Q:
    u_q = (q - 1/2) / Q
    (sn', cn', dn') = ellipj(u_q K', k'^2)                (real argument)
    sn_q = i sn'/cn',  cn_q = 1/cn',  dn_q = dn'/cn'      (Jacobi imaginary transform)
    w~_q    = -(2 sqrt(lambda_min) / (pi Q)) K' cn_q dn_q
    sigma_q^2 = lambda_min sn_q^2
  t_q = -sigma_q^2 > 0,  w_q = -w~_q > 0                  (Eq. contour_integral_quad_4)

so that K^{-1/2} ~= sum_q w_q (t_q I + K)^{-1}.  The 1/(pi i) factor of
Eq. contour_integral_quad_3 is already inside w~_q (Sec. 3 says the weights
absorb the normalising constant).
"""
from __future__ import annotations

import math

import numpy as np

from .elliptic import agm, ellipj


def quad_nodes(lmin: float, lmax: float, Q: int):
    """Weights ``w`` and shifts ``t`` (float64 arrays of length Q)."""
    if not (lmin > 0.0 and lmax >= lmin and Q >= 1):
        raise ValueError("need 0 < lmin <= lmax and Q >= 1")
    k2 = lmin / lmax
    k = math.sqrt(k2)
    kp2 = 1.0 - k2                      # k'^2, the parameter of the real-argument functions
    # K' = K(k') = pi / (2 AGM(1, sqrt(1 - k'^2))) = pi / (2 AGM(1, k)); using k
    # directly avoids the cancellation in 1 - k'^2 when kappa is large.
    Kp = math.pi / (2.0 * agm(1.0, k))
    w = np.empty(Q)
    t = np.empty(Q)
    for q in range(1, Q + 1):
        u = (q - 0.5) / Q
        snb, cnb, dnb = ellipj(u * Kp, kp2, mc=k2)
        sn_q = 1j * (snb / cnb)
        cn_q = 1.0 / cnb
        dn_q = dnb / cnb
        w_tilde = -(2.0 * math.sqrt(lmin) / (math.pi * Q)) * Kp * cn_q * dn_q
        sigma2 = lmin * sn_q * sn_q
        assert abs(np.imag(sigma2)) == 0.0
        w[q - 1] = -np.real(w_tilde)
        t[q - 1] = -np.real(sigma2)
    return w, t


def scalar_approx(lam, w, t):
    """sum_q w_q / (t_q + lambda): the quadrature applied to one eigenvalue."""
    lam = np.asarray(lam, dtype=np.float64)
    return np.sum(w[:, None] / (t[:, None] + lam.reshape(1, -1)), axis=0).reshape(lam.shape)
