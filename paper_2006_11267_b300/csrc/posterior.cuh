// Device pieces of posterior Thompson draws (Sec. 5 "Posterior Sampling for
// Bayesian Optimization", Eq. thompson_sample):
//     f* = mu* + COV*^{1/2} eps,   COV* = K** + jitter I - C C^T,
//     C = K*X (K_XX + sigma^2 I)^{-1/2},   mu* = m + C (K_XX + sigma^2 I)^{-1/2} (y - m).
#pragma once

#include "kernels.cuh"

namespace ciq {

// out[i * d + c] = X[i * d + c] / ls[c] (ARD lengthscales, device doubles).
cudaError_t launch_ard_scale(const float* X, int64_t N, int d, const double* ls, float* out, cudaStream_t st);

// FP64 kernel block: out[b * ldo + a] = s k(|x_a - z_b|) (+ diag on a == b
// when square), x = X1 (n1 points), z = X2 (n2 points), both already scaled
// (row-major, d floats each); rows a in [n1, ldo) are written as 0.
cudaError_t launch_kernel_block_f64(const float* X1, int64_t n1, const float* X2, int64_t n2, int d, int kt, double s,
                                    double diag, double* out, int64_t ldo, cudaStream_t st);

// mu[i] = m + sum_c Ct[c][i] a[c] (Ct: [n][ldc] FP32, a: n device doubles),
// rows [N, ldc) get m.
cudaError_t launch_posterior_mean(const float* Ct, int n, int64_t N, int64_t ldc, const double* a, double m, float* mu,
                                  cudaStream_t st);

// out[t * ldo + i] += mu[i] for i < N.
cudaError_t launch_add_mean(float* out, int64_t ldo, int64_t N, int T, const float* mu, cudaStream_t st);

}  // namespace ciq
