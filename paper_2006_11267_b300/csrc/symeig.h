// Symmetric eigendecomposition of a small dense matrix on the host (FP64).
//
// Used once per preconditioned solve for the R x R Gram matrix L^T L of the
// pivoted-Cholesky factor (R <= a few hundred).  Two classical steps:
//   1. Householder reduction to tridiagonal form, T = H^T A H, with the
//      orthogonal H accumulated (Golub and Van Loan, "Matrix Computations",
//      4th ed., Sec. 8.3.1);
//   2. implicit symmetric QR steps with the Wilkinson shift on the unreduced
//      blocks of T, deflating when an off-diagonal entry drops below machine
//      precision relative to its neighbours (Sec. 8.3.2-8.3.3); every Givens
//      rotation is applied to the columns of H, which become the eigenvectors.
// Plain C++ (no CUDA), header-only so that the host tests can build it alone.
#pragma once

#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

namespace ciq {
namespace symeig {

// A: n x n symmetric, column-major (A[i + j * n]); overwritten.
// w: n eigenvalues in ascending order; Z: n x n column-major, column k is the
// unit eigenvector of w[k].  Returns false if the QR iteration did not
// converge within 64 n sweeps (not expected for symmetric input).
inline bool eigh(int n, double* A, double* w, double* Z) {
    if (n <= 0) return true;
    auto a = [&](int i, int j) -> double& { return A[(size_t)i + (size_t)j * n]; };
    auto z = [&](int i, int j) -> double& { return Z[(size_t)i + (size_t)j * n]; };
    std::vector<double> d(n), e(n, 0.0);
    // Householder vectors stored below the subdiagonal of A (column k holds
    // v_k for the reflector I - beta_k v_k v_k^T acting on rows k+1..n-1).
    std::vector<double> beta(n, 0.0), p(n), v(n);
    for (int k = 0; k + 2 < n; ++k) {
        const int m = n - k - 1;                 // length of the reflected part
        double sigma = 0.0;
        for (int i = k + 2; i < n; ++i) sigma += a(i, k) * a(i, k);
        const double x0 = a(k + 1, k);
        if (sigma == 0.0) {                      // already zero below the subdiagonal
            beta[k] = 0.0;
            continue;
        }
        const double mu = std::sqrt(x0 * x0 + sigma);
        const double v0 = x0 <= 0.0 ? x0 - mu : -sigma / (x0 + mu);
        beta[k] = 2.0 * v0 * v0 / (sigma + v0 * v0);
        // v = (1, x[1:] / v0)
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = a(k + 1 + i, k) / v0;
        // p = beta A22 v,  w = p - (beta/2)(p^T v) v,  A22 -= v w^T + w v^T
        for (int i = 0; i < m; ++i) p[i] = 0.0;
        for (int j = 0; j < m; ++j) {
            const double vj = v[j];
            const double* col = &a(k + 1, k + 1 + j);
            for (int i = 0; i < m; ++i) p[i] += col[i] * vj;
        }
        for (int i = 0; i < m; ++i) p[i] *= beta[k];
        double pv = 0.0;
        for (int i = 0; i < m; ++i) pv += p[i] * v[i];
        const double c = 0.5 * beta[k] * pv;
        for (int i = 0; i < m; ++i) p[i] -= c * v[i];
        for (int j = 0; j < m; ++j)
            for (int i = 0; i < m; ++i) a(k + 1 + i, k + 1 + j) -= v[i] * p[j] + p[i] * v[j];
        a(k + 1, k) = mu;                        // H x = ||x|| e_1: the new subdiagonal entry
        for (int i = 1; i < m; ++i) a(k + 1 + i, k) = v[i];
    }
    for (int i = 0; i < n; ++i) d[i] = a(i, i);
    for (int i = 0; i + 1 < n; ++i) e[i] = a(i + 1, i);
    // H = H_0 H_1 ... H_{n-3}, accumulated backwards into Z.
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) z(i, j) = i == j ? 1.0 : 0.0;
    for (int k = n - 3; k >= 0; --k) {
        if (beta[k] == 0.0) continue;
        const int m = n - k - 1;
        v[0] = 1.0;
        for (int i = 1; i < m; ++i) v[i] = a(k + 1 + i, k);
        for (int j = k + 1; j < n; ++j) {
            double s = 0.0;
            for (int i = 0; i < m; ++i) s += v[i] * z(k + 1 + i, j);
            s *= beta[k];
            for (int i = 0; i < m; ++i) z(k + 1 + i, j) -= s * v[i];
        }
    }
    // Implicit symmetric QR with the Wilkinson shift.  The rotations depend on
    // the tridiagonal only, so they are recorded and applied to the columns
    // of Z afterwards, in order, by threads that each own a block of rows.
    struct Rot { int k; double c, s; };
    std::vector<Rot> rots;
    const double eps = 2.220446049250313e-16;
    int hi = n - 1;
    long sweeps = 0;
    while (hi > 0) {
        if (std::fabs(e[hi - 1]) <= eps * (std::fabs(d[hi - 1]) + std::fabs(d[hi]))) {
            e[hi - 1] = 0.0;
            --hi;
            continue;
        }
        int lo = hi - 1;
        while (lo > 0 && std::fabs(e[lo - 1]) > eps * (std::fabs(d[lo - 1]) + std::fabs(d[lo]))) --lo;
        if (++sweeps > 64L * n) return false;
        // Wilkinson shift from the trailing 2 x 2 block.
        const double dd = 0.5 * (d[hi - 1] - d[hi]);
        const double ee = e[hi - 1];
        const double den = dd + (dd >= 0.0 ? 1.0 : -1.0) * std::hypot(dd, ee);
        const double mu = d[hi] - (den != 0.0 ? ee * ee / den : 0.0);
        double x = d[lo] - mu, y = e[lo];
        for (int k = lo; k < hi; ++k) {
            // Givens rotation zeroing y against x.
            double c, s;
            if (y == 0.0) { c = 1.0; s = 0.0; }
            else if (std::fabs(y) > std::fabs(x)) { const double t = -x / y; s = 1.0 / std::sqrt(1.0 + t * t); c = s * t; }
            else { const double t = -y / x; c = 1.0 / std::sqrt(1.0 + t * t); s = c * t; }
            if (k > lo) e[k - 1] = c * x - s * y;
            // Apply G^T T G to rows/columns k, k+1 of the tridiagonal.
            const double dk = d[k], dk1 = d[k + 1], ek = e[k];
            const double c2 = c * c, s2 = s * s, cs = c * s;
            d[k] = c2 * dk - 2.0 * cs * ek + s2 * dk1;
            d[k + 1] = s2 * dk + 2.0 * cs * ek + c2 * dk1;
            e[k] = cs * (dk - dk1) + (c2 - s2) * ek;
            if (k + 1 < hi) {
                x = e[k];
                y = -s * e[k + 1];
                e[k + 1] *= c;
            }
            rots.push_back({k, c, s});
        }
    }
    // Row-major copy: a row of Z stays in cache while the whole rotation
    // sequence passes over it, four rows at a time.
    std::vector<double> Zr((size_t)n * n);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) Zr[(size_t)i * n + j] = z(i, j);
    auto apply_rows = [&](int r0, int r1) {
        int i = r0;
        for (; i + 4 <= r1; i += 4) {
            double* z0 = &Zr[(size_t)i * n];
            double* z1 = z0 + n;
            double* z2 = z1 + n;
            double* z3 = z2 + n;
            for (const Rot& g : rots) {
                const int k = g.k;
                const double a0 = z0[k], b0 = z0[k + 1], a1 = z1[k], b1 = z1[k + 1];
                const double a2 = z2[k], b2 = z2[k + 1], a3 = z3[k], b3 = z3[k + 1];
                z0[k] = g.c * a0 - g.s * b0; z0[k + 1] = g.s * a0 + g.c * b0;
                z1[k] = g.c * a1 - g.s * b1; z1[k + 1] = g.s * a1 + g.c * b1;
                z2[k] = g.c * a2 - g.s * b2; z2[k + 1] = g.s * a2 + g.c * b2;
                z3[k] = g.c * a3 - g.s * b3; z3[k + 1] = g.s * a3 + g.c * b3;
            }
        }
        for (; i < r1; ++i) {
            double* z0 = &Zr[(size_t)i * n];
            for (const Rot& g : rots) {
                const double a0 = z0[g.k], b0 = z0[g.k + 1];
                z0[g.k] = g.c * a0 - g.s * b0;
                z0[g.k + 1] = g.s * a0 + g.c * b0;
            }
        }
    };
    const int hw = (int)std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const int nth = n >= 128 ? std::min(hw, n / 16) : 1;
    if (nth <= 1) {
        apply_rows(0, n);
    } else {
        std::vector<std::thread> pool;
        const int per = ((n + nth - 1) / nth + 3) / 4 * 4;
        for (int t = 0; t < nth; ++t) {
            const int r0 = t * per, r1 = std::min(n, r0 + per);
            if (r0 < r1) pool.emplace_back(apply_rows, r0, r1);
        }
        for (auto& th : pool) th.join();
    }
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) z(i, j) = Zr[(size_t)i * n + j];
    // Ascending order (selection sort of the pairs; n is small).
    for (int i = 0; i < n; ++i) w[i] = d[i];
    for (int i = 0; i < n; ++i) {
        int k = i;
        for (int j = i + 1; j < n; ++j)
            if (w[j] < w[k]) k = j;
        if (k != i) {
            std::swap(w[i], w[k]);
            for (int r = 0; r < n; ++r) std::swap(z(r, i), z(r, k));
        }
    }
    return true;
}

}  // namespace symeig
}  // namespace ciq
