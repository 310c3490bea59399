// Backward pass of msMINRES-CIQ (Sec. 3.4, Eq. ciq_deriv).
//
// Differentiating each quadrature term with the nodes fixed gives
//   dL/dtheta = sum_q c_q y_q^T (dK/dtheta) x_q,
// x_q = (t_q + K)^{-1} b, y_q = (t_q + K)^{-1} g (g = dL/da), c_q = -w_q for
// K^{-1/2} b and +w_q t_q for K^{1/2} b (identity form).  The solve runs on
// the 2T columns [B | G] in the stored-basis form, so x_q and y_q of every
// column are V_c y_q(.) with the per-shift coefficients the back-substitution
// records; this file forms them and the three contractions:
//   * basis_solutions: Xq[q][c] = sum_j y_q(j) q_j of column c, four shifts
//     per pass over the basis;
//   * vjp_bilinear: sum over 64 x 64 tiles (i, j) of K of
//     A_ij = sum_{c<T,q} c_q y_qc[i] x_qc[j] times dk/dl (scaled by s) and
//     times k/s, with kernel values from coordinate differences of the
//     scaled points (RBF dk/dl = k r~^2 / l, Matern-5/2 dk/dl = s (z^2 / 3l)
//     (1 + z) e^{-z}, r~ = r / l, z = sqrt(5) r~), per-block FP64 partials;
//   * vjp_dots: sum_{c<T,q} c_q y_qc . x_qc (dK/dsigma^2 = I);
//   * vjp_reduce: the partials summed in a fixed order.
#include <math.h>

#include "krylov.cuh"

namespace ciq {
namespace {

constexpr int kVT = 64;          // tile edge of the bilinear pass
constexpr int kQG = 4;           // shifts per pass of basis_solutions

__device__ __forceinline__ double vjp_coef(const KrylovState<float>& s, int q) {
    const double w = s.nodes[kNodeW + q], t = s.nodes[kNodeT + q];
    return s.op == kOpInvSqrt ? -w : w * t;
}

// One block per (row chunk, column): shifts q0..q0+3 of column c.
__global__ void __launch_bounds__(256) basis_solutions_kernel(KrylovState<float> s, float* Xq, int q0) {
    __shared__ float cf[256][kQG];
    const int k = blockIdx.x, c = blockIdx.y, tid = threadIdx.x;
    const int T = s.T, Q = s.Q;
    const int J = s.iters[c];
    const int64_t vs = (int64_t)T * s.Npad;
    const int64_t col = (int64_t)c * s.Npad;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    const int nq = min(kQG, Q - q0);
    for (int64_t base = i0; base < i1; base += 256) {
        const int64_t i = base + tid;
        float acc[kQG] = {0.f, 0.f, 0.f, 0.f};
        for (int jb = 1; jb <= J; jb += 256) {
            const int nj = min(256, J - jb + 1);
            __syncthreads();
            if (tid < nj)
                for (int u = 0; u < kQG; ++u)
                    cf[tid][u] = u < nq ? (float)s.ycoef[((int64_t)(jb + tid) * Q + q0 + u) * T + c] : 0.f;
            __syncthreads();
            if (i < i1) {
                const float* vp = s.basis + (int64_t)jb * vs + col + i;
#pragma unroll 4
                for (int u = 0; u < nj; ++u) {
                    const float v = vp[(int64_t)u * vs];
#pragma unroll
                    for (int e = 0; e < kQG; ++e) acc[e] = fmaf(cf[u][e], v, acc[e]);
                }
            }
        }
        if (i < i1)
            for (int e = 0; e < nq; ++e) Xq[((int64_t)(q0 + e) * T + c) * s.Npad + i] = acc[e];
    }
}

// One block per 64 x 64 tile of K; 256 threads, a 4 x 4 block of entries
// each (register-tiled rank-R update, two 16-byte shared loads per 16 FMAs).
__global__ void __launch_bounds__(256) vjp_bilinear_kernel(KrylovState<float> s, const float* Xp, int dp, int kt,
                                                           float inv_l, float sc, const float* Xq, int Tb,
                                                           double* part) {
    constexpr int RC = 16;                                // (shift, column) pairs per shared-memory panel
    __shared__ __align__(16) float Ys[RC][kVT];
    __shared__ __align__(16) float Xs[RC][kVT];
    __shared__ float Pi[kVT][17], Pj[kVT][17];
    __shared__ double red[8][2];
    __shared__ float cqs[CIQ_MAX_Q];
    const int nt = (int)(s.Npad / kVT);
    const int bi = blockIdx.x % nt, bj = blockIdx.x / nt;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    const int64_t i0 = (int64_t)bi * kVT, j0 = (int64_t)bj * kVT;
    const int Q = s.Q, T2 = s.T;
    for (int e = tid; e < kVT * dp; e += 256) {
        const int r = e / dp, k = e % dp;
        Pi[r][k] = Xp[(i0 + r) * dp + k];
        Pj[r][k] = Xp[(j0 + r) * dp + k];
    }
    if (tid < Q) cqs[tid] = (float)vjp_coef(s, tid);
    float A[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) A[a][b] = 0.f;
    const int R = Q * Tb;                                 // (shift, column) pairs
    for (int r0 = 0; r0 < R; r0 += RC) {
        __syncthreads();
        for (int e = tid; e < RC * kVT; e += 256) {
            const int rr = e / kVT, row = e % kVT, r = r0 + rr;     // consecutive threads: consecutive rows
            float yv = 0.f, xv = 0.f;
            if (r < R) {
                const int q = r / Tb, c = r % Tb;
                yv = cqs[q] * Xq[((int64_t)q * T2 + Tb + c) * s.Npad + i0 + row];
                xv = Xq[((int64_t)q * T2 + c) * s.Npad + j0 + row];
            }
            Ys[rr][row] = yv;
            Xs[rr][row] = xv;
        }
        __syncthreads();
#pragma unroll
        for (int rr = 0; rr < RC; ++rr) {
            const float4 y = *reinterpret_cast<const float4*>(&Ys[rr][4 * ty]);
            const float4 x = *reinterpret_cast<const float4*>(&Xs[rr][4 * tx]);
            const float ya[4] = {y.x, y.y, y.z, y.w}, xa[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
            for (int a = 0; a < 4; ++a)
#pragma unroll
                for (int b = 0; b < 4; ++b) A[a][b] = fmaf(ya[a], xa[b], A[a][b]);
        }
    }
    // Kernel values of this thread's 16 entries, from coordinate differences.
    float gl = 0.f, gs = 0.f;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            float r2 = 0.f;
            for (int k = 0; k < dp; ++k) {
                const float df = Pi[4 * ty + a][k] - Pj[4 * tx + b][k];
                r2 = fmaf(df, df, r2);
            }
            float kv, dl;
            if (kt == CIQ_RBF) {
                kv = expf(-0.5f * r2);
                dl = sc * kv * r2 * inv_l;
            } else {
                const float z = sqrtf(5.f * r2);
                const float ez = expf(-z);
                kv = (1.f + z + z * z * (1.f / 3.f)) * ez;
                dl = sc * (z * z * (1.f / 3.f) * inv_l) * (1.f + z) * ez;
            }
            gl = fmaf(dl, A[a][b], gl);
            gs = fmaf(kv, A[a][b], gs);
        }
    }
    double dgl = warp_sum((double)gl), dgs = warp_sum((double)gs);
    if ((tid & 31) == 0) { red[tid >> 5][0] = dgl; red[tid >> 5][1] = dgs; }
    __syncthreads();
    if (tid == 0) {
        double a = 0.0, b = 0.0;
        for (int w = 0; w < 8; ++w) { a += red[w][0]; b += red[w][1]; }
        part[2 * (int64_t)blockIdx.x] = a;
        part[2 * (int64_t)blockIdx.x + 1] = b;
    }
}

// One block per (shift, column of B): c_q y_qc . x_qc.
__global__ void __launch_bounds__(256) vjp_dots_kernel(KrylovState<float> s, const float* Xq, int Tb, double* part) {
    __shared__ double red[8];
    const int q = blockIdx.x / Tb, c = blockIdx.x % Tb, tid = threadIdx.x;
    const float* x = Xq + ((int64_t)q * s.T + c) * s.Npad;
    const float* y = Xq + ((int64_t)q * s.T + Tb + c) * s.Npad;
    double acc = 0.0;
    for (int64_t i = tid; i < s.Npad; i += 256) acc += (double)x[i] * (double)y[i];
    acc = warp_sum(acc);
    if ((tid & 31) == 0) red[tid >> 5] = acc;
    __syncthreads();
    if (tid == 0) {
        double a = 0.0;
        for (int w = 0; w < 8; ++w) a += red[w];
        part[blockIdx.x] = vjp_coef(s, q) * a;
    }
}

// grad[0..2] from the partials, in a fixed order (one warp).
__global__ void vjp_reduce_kernel(const double* bil, int64_t nbil, const double* dots, int ndots, double* grad) {
    const int lane = threadIdx.x;
    double a[4] = {0.0, 0.0, 0.0, 0.0}, b[4] = {0.0, 0.0, 0.0, 0.0}, c = 0.0;
    int64_t e = lane;
    for (; e + 96 < nbil; e += 128)                      // four independent chains per lane
        for (int u = 0; u < 4; ++u) { a[u] += bil[2 * (e + 32 * u)]; b[u] += bil[2 * (e + 32 * u) + 1]; }
    for (; e < nbil; e += 32) { a[0] += bil[2 * e]; b[0] += bil[2 * e + 1]; }
    for (int d = lane; d < ndots; d += 32) c += dots[d];
    double sa = (a[0] + a[1]) + (a[2] + a[3]), sb = (b[0] + b[1]) + (b[2] + b[3]);
    sa = warp_sum(sa);
    sb = warp_sum(sb);
    c = warp_sum(c);
    if (lane == 0) { grad[0] = sa; grad[1] = sb; grad[2] = c; }
}

}  // namespace

int64_t vjp_partials(int64_t Npad, int T, int Q) {
    const int64_t nt = Npad / kVT;
    return 2 * nt * nt + (int64_t)Q * T;
}

cudaError_t launch_vjp(const KrylovState<float>& s, const float* Xp, int dp, int kt, double lengthscale,
                       double outputscale, float* Xq, double* part, double* grad, cudaStream_t st) {
    if (s.T % 2 != 0 || !s.ycoef || !s.basis || s.Npad % kVT != 0 || dp > 16) return cudaErrorInvalidValue;
    const int Tb = s.T / 2;
    for (int q0 = 0; q0 < s.Q; q0 += kQG)
        basis_solutions_kernel<<<dim3(s.nchunks, s.T), 256, 0, st>>>(s, Xq, q0);
    const int64_t nt = s.Npad / kVT;
    double* bil = part;
    double* dots = part + 2 * nt * nt;
    vjp_bilinear_kernel<<<(unsigned)(nt * nt), 256, 0, st>>>(s, Xp, dp, kt, (float)(1.0 / lengthscale),
                                                            (float)outputscale, Xq, Tb, bil);
    vjp_dots_kernel<<<s.Q * Tb, 256, 0, st>>>(s, Xq, Tb, dots);
    vjp_reduce_kernel<<<1, 32, 0, st>>>(bil, nt * nt, dots, s.Q * Tb, grad);
    return cudaGetLastError();
}

}  // namespace ciq
