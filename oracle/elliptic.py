"""Complete elliptic integral and Jacobi elliptic functions in FP64.

The quadrature of App. B (Eq. quad_points_and_locations, Algorithm
"quadrature") needs K'(k) = K(k') and sn, cn, dn at parameter m' = k'^2 =
1 - k^2.  The paper calls SciPy's ``ellipke``/``ellipj``; the oracle
implements the arithmetic-geometric mean (AGM) methods of Abramowitz and
Stegun instead, so that it can be checked against SciPy:

* A&S 17.6: K(m) = pi / (2 AGM(1, sqrt(1 - m))).
* A&S 16.4: descending Landen / AGM scheme for sn, cn, dn.

Both take the complementary parameter ``mc = 1 - m`` explicitly: for an
ill-conditioned kernel matrix m' = 1 - lambda_min/lambda_max is within
1e-8 of 1, and forming 1 - m' would cancel.
"""
from __future__ import annotations

import math

EPS = 2.0 ** -53


def agm(a: float, b: float) -> float:
    """Arithmetic-geometric mean of two non-negative numbers."""
    for _ in range(100):
        if abs(a - b) <= 4 * EPS * a:
            break
        a, b = 0.5 * (a + b), math.sqrt(a * b)
    return 0.5 * (a + b)


def ellipk_mc(mc: float) -> float:
    """K(m) given the complementary parameter ``mc = 1 - m`` (A&S 17.6)."""
    if mc <= 0.0:
        return math.inf
    return math.pi / (2.0 * agm(1.0, math.sqrt(mc)))


def ellipj(u: float, m: float, mc: float | None = None):
    """(sn, cn, dn)(u | m) by the AGM scheme of A&S 16.4.

    a_0 = 1, b_0 = sqrt(mc), c_0 = sqrt(m); a_n, b_n, c_n by the AGM step until
    c_N is negligible; phi_N = 2^N a_N u; phi_{n-1} = (phi_n + asin(c_n sin(phi_n)
    / a_n)) / 2; then sn = sin phi_0, cn = cos phi_0, dn = sqrt(mc + m cn^2).
    """
    if mc is None:
        mc = 1.0 - m
    if m < 0.0 or mc < 0.0:
        raise ValueError("parameter must lie in [0, 1]")
    if m == 0.0:
        return math.sin(u), math.cos(u), 1.0
    if mc == 0.0:
        s = 1.0 / math.cosh(u)
        return math.tanh(u), s, s
    a = [1.0]
    c = [math.sqrt(m)]
    b = math.sqrt(mc)
    while abs(c[-1]) > EPS * a[-1] and len(a) < 64:
        an, bn, cn = 0.5 * (a[-1] + b), math.sqrt(a[-1] * b), 0.5 * (a[-1] - b)
        a.append(an)
        c.append(cn)
        b = bn
    nsteps = len(a) - 1
    phi = (2.0 ** nsteps) * a[-1] * u
    phis = [phi]
    for n in range(nsteps, 0, -1):
        phi = 0.5 * (phi + math.asin(c[n] * math.sin(phi) / a[n]))
        phis.append(phi)
    phi0 = phis[-1]
    sn = math.sin(phi0)
    cn = math.cos(phi0)
    # dn^2 = 1 - m sn^2 = mc + m cn^2 (A&S 16.9.1): a sum of non-negative
    # terms, accurate near the quarter period where A&S 16.4.3's
    # cos(phi_0) / cos(phi_1 - phi_0) becomes 0/0.
    dn = math.sqrt(mc + m * cn * cn)
    return sn, cn, dn
