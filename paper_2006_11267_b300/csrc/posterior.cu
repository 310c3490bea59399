// Posterior Thompson draws: ARD scaling, FP64 kernel blocks of the training
// set, the posterior mean, and the mean added to the draws.  The correction
// C = K*X W with W = (K_XX + sigma^2 I)^{-1/2} (host eigendecomposition, FP64)
// is formed by launch_product_f64 (precond.cu), and the draws run
// msMINRES-CIQ on K** + jitter I with the low-rank correction -C C^T applied
// in every MVM's epilogue (launch_lowrank_lanczos).
#include "posterior.cuh"

namespace ciq {

namespace {

__global__ void ard_scale_kernel(const float* X, int64_t N, int d, const double* ls, float* out) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= N * d) return;
    out[e] = (float)((double)X[e] / ls[e % d]);
}

// One thread per output entry; column b of the block is contiguous.
__global__ void kernel_block_f64(const float* X1, int64_t n1, const float* X2, int64_t n2, int d, int kt, double s,
                                 double diag, double* out, int64_t ldo) {
    const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t b = blockIdx.y;
    if (a >= ldo || b >= n2) return;
    double v = 0.0;
    if (a < n1) {
        double r2 = 0.0;
        for (int c = 0; c < d; ++c) {
            const double df = (double)X1[a * d + c] - (double)X2[b * d + c];
            r2 = fma(df, df, r2);
        }
        v = kt == CIQ_RBF ? kernel_value<CIQ_RBF>(r2, s) : kernel_value<CIQ_MATERN52>(r2, s);
        if (a == b && X1 == X2) v += diag;
    }
    out[b * ldo + a] = v;
}

__global__ void posterior_mean_kernel(const float* Ct, int n, int64_t N, int64_t ldc, const double* a, double m,
                                      float* mu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= ldc) return;
    double s = m;
    if (i < N)
        for (int c = 0; c < n; ++c) s = fma((double)Ct[(int64_t)c * ldc + i], a[c], s);
    mu[i] = (float)s;
}

__global__ void add_mean_kernel(float* out, int64_t ldo, int64_t N, const float* mu) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) out[(int64_t)blockIdx.y * ldo + i] += mu[i];
}

}  // namespace

cudaError_t launch_ard_scale(const float* X, int64_t N, int d, const double* ls, float* out, cudaStream_t st) {
    const int64_t n = N * d;
    if (n > 0) ard_scale_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(X, N, d, ls, out);
    return cudaGetLastError();
}

cudaError_t launch_kernel_block_f64(const float* X1, int64_t n1, const float* X2, int64_t n2, int d, int kt, double s,
                                    double diag, double* out, int64_t ldo, cudaStream_t st) {
    if (n2 < 1 || ldo < 1) return cudaSuccess;
    kernel_block_f64<<<dim3((unsigned)((ldo + 127) / 128), (unsigned)n2), 128, 0, st>>>(X1, n1, X2, n2, d, kt, s,
                                                                                        diag, out, ldo);
    return cudaGetLastError();
}

cudaError_t launch_posterior_mean(const float* Ct, int n, int64_t N, int64_t ldc, const double* a, double m, float* mu,
                                  cudaStream_t st) {
    posterior_mean_kernel<<<(unsigned)((ldc + 255) / 256), 256, 0, st>>>(Ct, n, N, ldc, a, m, mu);
    return cudaGetLastError();
}

cudaError_t launch_add_mean(float* out, int64_t ldo, int64_t N, int T, const float* mu, cudaStream_t st) {
    if (T < 1 || N < 1) return cudaSuccess;
    add_mean_kernel<<<dim3((unsigned)((N + 255) / 256), (unsigned)T), 256, 0, st>>>(out, ldo, N, mu);
    return cudaGetLastError();
}

}  // namespace ciq
