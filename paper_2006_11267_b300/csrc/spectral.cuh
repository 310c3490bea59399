// FP64 scalar routines shared by the host entry point ciq_quad_nodes and the
// device kernel that turns Lanczos coefficients into quadrature nodes, so
// that the whole solve can run without a host round trip.
//
//  * complete elliptic integral by the arithmetic-geometric mean (A&S 17.6)
//  * Jacobi sn, cn, dn by the descending AGM scheme (A&S 16.4), with
//    dn = sqrt(mc + m cn^2) (A&S 16.9.1), accurate near the quarter period
//  * Hale-Higham-Trefethen nodes for K^{-1/2} (Eq. quad_points_and_locations,
//    sign flip of Eq. contour_integral_quad_4), with the definition
//    k'^2 = 1 - k^2 (the printed sqrt(1 - k^2) contradicts it)
//  * extreme eigenvalues of a symmetric tridiagonal matrix by Sturm-count
//    bisection (Ritz values of the Lanczos T_J, App. B.2)
#pragma once

#include <math.h>

#include "common.cuh"

namespace ciq {

CIQ_HD double agm(double a, double b) {
    for (int it = 0; it < 64; ++it) {
        if (fabs(a - b) <= 8.881784197001252e-16 * a) break;
        double an = 0.5 * (a + b);
        b = sqrt(a * b);
        a = an;
    }
    return 0.5 * (a + b);
}

// sn, cn, dn of u at parameter m, given mc = 1 - m separately.
CIQ_HD void jacobi_sncndn(double u, double m, double mc, double* sn, double* cn, double* dn) {
    if (m == 0.0) { *sn = sin(u); *cn = cos(u); *dn = 1.0; return; }
    if (mc == 0.0) { double s = 1.0 / cosh(u); *sn = tanh(u); *cn = s; *dn = s; return; }
    double a[40], c[40];
    a[0] = 1.0;
    c[0] = sqrt(m);
    double b = sqrt(mc);
    int n = 0;
    while (fabs(c[n]) > 1.1102230246251565e-16 * a[n] && n < 38) {
        double an = 0.5 * (a[n] + b);
        double cn1 = 0.5 * (a[n] - b);
        b = sqrt(a[n] * b);
        ++n;
        a[n] = an;
        c[n] = cn1;
    }
    double phi = ldexp(a[n] * u, n);
    for (int k = n; k >= 1; --k) phi = 0.5 * (phi + asin(c[k] * sin(phi) / a[k]));
    *sn = sin(phi);
    *cn = cos(phi);
    *dn = sqrt(mc + m * (*cn) * (*cn));
}

// Returns 0 on success, -1 on bad arguments.
CIQ_HD int quad_nodes(double lmin, double lmax, int Q, double* w, double* t) {
    if (!(lmin > 0.0) || !(lmax >= lmin) || Q < 1 || Q > CIQ_MAX_Q) return -1;
    const double pi = 3.141592653589793;
    double k2 = lmin / lmax;                 // k^2
    double k = sqrt(k2);
    double kp2 = 1.0 - k2;                   // k'^2 (parameter of the real-argument functions)
    double Kp = pi / (2.0 * agm(1.0, k));    // K'(k) = K(k') = pi / (2 AGM(1, k))
    double pref = 2.0 * sqrt(lmin) / (pi * (double)Q);
    for (int q = 1; q <= Q; ++q) {
        double u = ((double)q - 0.5) / (double)Q;
        double snb, cnb, dnb;
        jacobi_sncndn(u * Kp, kp2, k2, &snb, &cnb, &dnb);
        // Imaginary transform: sn(iuK'|k) = i snb/cnb, cn = 1/cnb, dn = dnb/cnb.
        // sigma^2 = lmin sn^2 = -lmin (snb/cnb)^2; w~ = -pref K' cn dn.
        double ratio = snb / cnb;
        t[q - 1] = lmin * ratio * ratio;                 // t_q = -sigma_q^2
        w[q - 1] = pref * Kp * dnb / (cnb * cnb);        // w_q = -w~_q
    }
    return 0;
}

// Number of eigenvalues of tridiag(off; diag; off) strictly below x.
// off[k] couples rows k-1 and k (off[0] unused).
CIQ_HD int sturm_count(const double* diag, const double* off, int J, double x) {
    int cnt = 0;
    double q = diag[0] - x;
    if (q < 0.0) ++cnt;
    for (int k = 1; k < J; ++k) {
        if (q == 0.0) q = 1e-300;
        q = (diag[k] - x) - off[k] * off[k] / q;
        if (q < 0.0) ++cnt;
    }
    return cnt;
}

// Smallest (want_max = false) or largest eigenvalue by bisection.
CIQ_HD double tridiag_extreme(const double* diag, const double* off, int J, bool want_max) {
    double lo = diag[0], hi = diag[0];
    for (int k = 0; k < J; ++k) {
        double r = (k > 0 ? fabs(off[k]) : 0.0) + (k + 1 < J ? fabs(off[k + 1]) : 0.0);
        lo = fmin(lo, diag[k] - r);
        hi = fmax(hi, diag[k] + r);
    }
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        int c = sturm_count(diag, off, J, mid);
        bool go_left = want_max ? (c == J) : (c >= 1);
        if (go_left) hi = mid; else lo = mid;
    }
    return 0.5 * (lo + hi);
}

}  // namespace ciq
