// Learned spectral-bound predictor: features, training and inference kernels.
//
// The paper has no learned component.  This small regression network maps a
// problem's description to what the Lanczos pre-pass (App. B.2) and msMINRES
// (App. C) would report -- log theta_min, log theta_max and log of the
// iteration count -- so that a batch can skip the pre-pass (bounds given per
// problem) and fall back to it where the solve shows the bounds were wrong.
//
//   inputs (38): log N, d, kernel type, log lengthscale, log outputscale,
//                log max(sigma^2, 1e-12), per-coordinate mean and population
//                variance of X for coordinates 0..15 (0 past d);
//   network:     standardised inputs -> 64 tanh -> 64 tanh -> 3 linear,
//                outputs de-standardised;
//   loss:        mean over samples and outputs of the squared standardised error;
//   training:    Adam with bias correction (0.9, 0.999, 1e-8); minibatch
//                index k of step t is floor(u n), u the splitmix64 uniform
//                number (t - 1) * batch + k of the seed.
//
// Parameter layout (floats): input means [0,38), input standard deviations
// [38,76), output means [76,79), output standard deviations [79,82), then
// W1 (38 x 64, input-major), b1, W2 (64 x 64), b2, W3 (64 x 3), b3.
//
// Training runs in one CTA (the network is 6.9k parameters; a step is a few
// microseconds of work) that loops over all Adam steps with the parameters
// and Adam moments resident in shared memory; each minibatch is processed in
// chunks of 32 samples whose activations and deltas stay in shared memory.
#include <cuda_bf16.h>
#include <math.h>

#include "common.cuh"
#include "mlp.cuh"

namespace ciq {

namespace {

constexpr int kCB = 32;                 // samples per chunk
constexpr int kLD0 = kMlpIn + 1;        // padded row strides of the chunk arrays
constexpr int kLDH = kMlpHid + 1;

__device__ __forceinline__ double mlp_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

// Shared-memory working set of one chunk.
struct Chunk {
    float* z0;    // [kCB][kLD0] standardised inputs
    float* h1;    // [kCB][kLDH]
    float* h2;    // [kCB][kLDH]
    float* ds;    // [kCB][3]    d loss / d standardised output
    float* da2;   // [kCB][kLDH] d loss / d pre-activation 2
    float* da1;   // [kCB][kLDH] d loss / d pre-activation 1
};

__device__ __forceinline__ size_t chunk_floats() { return (size_t)kCB * (kLD0 + 4 * kLDH + 3); }

__device__ __forceinline__ Chunk chunk_view(float* base) {
    Chunk c;
    c.z0 = base;
    c.h1 = c.z0 + kCB * kLD0;
    c.h2 = c.h1 + kCB * kLDH;
    c.da2 = c.h2 + kCB * kLDH;
    c.da1 = c.da2 + kCB * kLDH;
    c.ds = c.da1 + kCB * kLDH;
    return c;
}

// Forward and backward over `cnt` samples (rows idx[0..cnt) of F, Y) with
// parameters w (shared); adds the gradient to g (shared, trained entries)
// and the sum of squared standardised errors to *sq.  inv_m = 1 / (3 x
// minibatch size).  256 threads.
__device__ void chunk_fwd_bwd(const float* w, float* g, const Chunk& c, const float* F, const float* Y,
                              const int* idx, int cnt, float inv_m, float* sq) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const float* fmu = w;
    const float* fsd = w + kMlpIn;
    const float* ymu = w + 2 * kMlpIn;
    const float* ysd = ymu + kMlpOut;
    const float* W1 = w + kMlpOffW1;
    const float* b1 = w + kMlpOffB1;
    const float* W2 = w + kMlpOffW2;
    const float* b2 = w + kMlpOffB2;
    const float* W3 = w + kMlpOffW3;
    const float* b3 = w + kMlpOffB3;
    for (int e = tid; e < kCB * kMlpIn; e += 256) {
        const int s = e / kMlpIn, i = e % kMlpIn;
        c.z0[s * kLD0 + i] = s < cnt ? (F[(int64_t)idx[s] * kMlpIn + i] - fmu[i]) / fsd[i] : 0.f;
    }
    __syncthreads();
    for (int e = tid; e < kCB * kMlpHid; e += 256) {
        const int s = e / kMlpHid, h = e % kMlpHid;
        float a = b1[h];
        for (int i = 0; i < kMlpIn; ++i) a = fmaf(c.z0[s * kLD0 + i], W1[i * kMlpHid + h], a);
        c.h1[s * kLDH + h] = tanhf(a);
    }
    __syncthreads();
    for (int e = tid; e < kCB * kMlpHid; e += 256) {
        const int s = e / kMlpHid, h = e % kMlpHid;
        float a = b2[h];
        for (int k = 0; k < kMlpHid; ++k) a = fmaf(c.h1[s * kLDH + k], W2[k * kMlpHid + h], a);
        c.h2[s * kLDH + h] = tanhf(a);
    }
    __syncthreads();
    float part = 0.f;
    if (tid < kCB * kMlpOut) {
        const int s = tid / kMlpOut, o = tid % kMlpOut;
        float a = b3[o];
        for (int h = 0; h < kMlpHid; ++h) a = fmaf(c.h2[s * kLDH + h], W3[h * kMlpOut + o], a);
        float r = 0.f;
        if (s < cnt) r = a - (Y[(int64_t)idx[s] * kMlpOut + o] - ymu[o]) / ysd[o];
        part = r * r;
        c.ds[s * kMlpOut + o] = 2.f * r * inv_m;
    }
    part = warp_sum(part);
    if (lane == 0 && warp < (kCB * kMlpOut + 31) / 32) atomicAdd(sq, part);
    __syncthreads();
    // Output layer gradient and delta of layer 2.
    if (tid < kMlpHid * kMlpOut) {
        const int h = tid / kMlpOut, o = tid % kMlpOut;
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a = fmaf(c.h2[s * kLDH + h], c.ds[s * kMlpOut + o], a);
        g[kMlpOffW3 + h * kMlpOut + o] += a;
    } else if (tid < kMlpHid * kMlpOut + kMlpOut) {
        const int o = tid - kMlpHid * kMlpOut;
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a += c.ds[s * kMlpOut + o];
        g[kMlpOffB3 + o] += a;
    }
    for (int e = tid; e < kCB * kMlpHid; e += 256) {
        const int s = e / kMlpHid, h = e % kMlpHid;
        float a = 0.f;
#pragma unroll
        for (int o = 0; o < kMlpOut; ++o) a = fmaf(c.ds[s * kMlpOut + o], W3[h * kMlpOut + o], a);
        const float hv = c.h2[s * kLDH + h];
        c.da2[s * kLDH + h] = a * (1.f - hv * hv);
    }
    __syncthreads();
    // Layer 2 gradient; delta of layer 1 (lane = sample, so the padded
    // strides keep shared-memory reads conflict-free).
    for (int e = tid; e < kMlpHid * kMlpHid; e += 256) {
        const int k = e / kMlpHid, h = e % kMlpHid;
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a = fmaf(c.h1[s * kLDH + k], c.da2[s * kLDH + h], a);
        g[kMlpOffW2 + k * kMlpHid + h] += a;
    }
    if (tid < kMlpHid) {
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a += c.da2[s * kLDH + tid];
        g[kMlpOffB2 + tid] += a;
    }
    for (int k = warp; k < kMlpHid; k += 8) {
        const int s = lane;
        float a = 0.f;
        for (int h = 0; h < kMlpHid; ++h) a = fmaf(c.da2[s * kLDH + h], W2[k * kMlpHid + h], a);
        const float hv = c.h1[s * kLDH + k];
        c.da1[s * kLDH + k] = a * (1.f - hv * hv);
    }
    __syncthreads();
    for (int e = tid; e < kMlpIn * kMlpHid; e += 256) {
        const int i = e / kMlpHid, k = e % kMlpHid;
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a = fmaf(c.z0[s * kLD0 + i], c.da1[s * kLDH + k], a);
        g[kMlpOffW1 + i * kMlpHid + k] += a;
    }
    if (tid < kMlpHid) {
        float a = 0.f;
        for (int s = 0; s < kCB; ++s) a += c.da1[s * kLDH + tid];
        g[kMlpOffB1 + tid] += a;
    }
    __syncthreads();
}

size_t train_smem_bytes() { return sizeof(float) * (4 * (size_t)kMlpParams + (size_t)kCB * (kLD0 + 4 * kLDH + 3) + 8) + sizeof(int) * kCB; }
size_t grad_smem_bytes() { return sizeof(float) * (2 * (size_t)kMlpParams + (size_t)kCB * (kLD0 + 4 * kLDH + 3) + 8) + sizeof(int) * kCB; }

// Full-batch loss and gradient: block b takes samples 32b .. 32b+31 and adds
// its FP32 chunk sums into the FP64 totals.
__global__ void __launch_bounds__(256) mlp_grad_kernel(const float* theta, const float* F, const float* Y, int n,
                                                       double* loss, double* grad) {
    extern __shared__ float smem[];
    float* w = smem;
    float* g = w + kMlpParams;
    float* sq = g + kMlpParams;
    float* cbase = sq + 8;
    int* idx = reinterpret_cast<int*>(cbase + chunk_floats());
    for (int e = threadIdx.x; e < kMlpParams; e += 256) { w[e] = theta[e]; g[e] = 0.f; }
    if (threadIdx.x == 0) *sq = 0.f;
    const int s0 = blockIdx.x * kCB;
    const int cnt = min(kCB, n - s0);
    if (threadIdx.x < kCB) idx[threadIdx.x] = s0 + min((int)threadIdx.x, cnt - 1);
    __syncthreads();
    chunk_fwd_bwd(w, g, chunk_view(cbase), F, Y, idx, cnt, 1.f / (3.f * (float)n), sq);
    for (int e = kMlpOffW1 + threadIdx.x; e < kMlpParams; e += 256) atomicAdd(&grad[e], (double)g[e]);
    if (threadIdx.x == 0) atomicAdd(loss, (double)*sq / (3.0 * (double)n));
}

// `steps` Adam steps in one CTA; theta, m, v updated in place in global memory.
__global__ void __launch_bounds__(256) mlp_train_kernel(float* theta, float* adam_m, float* adam_v, const float* F,
                                                        const float* Y, int n, int steps, int batch, float lr,
                                                        uint64_t seed, int first_step, float* losses) {
    extern __shared__ float smem[];
    float* w = smem;
    float* g = w + kMlpParams;
    float* m = g + kMlpParams;
    float* v = m + kMlpParams;
    float* sq = v + kMlpParams;
    float* cbase = sq + 8;
    int* idx = reinterpret_cast<int*>(cbase + chunk_floats());
    const Chunk c = chunk_view(cbase);
    for (int e = threadIdx.x; e < kMlpParams; e += 256) {
        w[e] = theta[e];
        m[e] = adam_m[e];
        v[e] = adam_v[e];
    }
    __syncthreads();
    const float inv_m = 1.f / (3.f * (float)batch);
    for (int t = first_step; t < first_step + steps; ++t) {
        for (int e = threadIdx.x; e < kMlpParams; e += 256) g[e] = 0.f;
        if (threadIdx.x == 0) *sq = 0.f;
        __syncthreads();
        for (int s0 = 0; s0 < batch; s0 += kCB) {
            const int cnt = min(kCB, batch - s0);
            if (threadIdx.x < kCB) {
                const int k = s0 + min((int)threadIdx.x, cnt - 1);
                const double u = mlp_uniform(seed, (uint64_t)(t - 1) * (uint64_t)batch + (uint64_t)k);
                idx[threadIdx.x] = min((int)floor(u * (double)n), n - 1);
            }
            __syncthreads();
            chunk_fwd_bwd(w, g, c, F, Y, idx, cnt, inv_m, sq);
        }
        const float bc1 = (float)(1.0 - pow(0.9, (double)t));
        const float bc2 = (float)(1.0 - pow(0.999, (double)t));
        for (int e = kMlpOffW1 + threadIdx.x; e < kMlpParams; e += 256) {
            const float ge = g[e];
            const float me = 0.9f * m[e] + 0.1f * ge;
            const float ve = 0.999f * v[e] + 0.001f * ge * ge;
            m[e] = me;
            v[e] = ve;
            w[e] -= lr * (me / bc1) / (sqrtf(ve / bc2) + 1e-8f);
        }
        if (threadIdx.x == 0 && losses) losses[t - first_step] = *sq * inv_m;
        __syncthreads();
    }
    for (int e = threadIdx.x; e < kMlpParams; e += 256) {
        theta[e] = w[e];
        adam_m[e] = m[e];
        adam_v[e] = v[e];
    }
}

__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

// One warp per sample; weights (BF16-rounded when bf16 != 0) in shared memory.
__global__ void __launch_bounds__(256) mlp_predict_kernel(const float* theta, const float* F, int n, float* out,
                                                          int bf16) {
    __shared__ float w[kMlpParams];
    __shared__ float z0[8][kMlpIn], h1[8][kMlpHid], h2[8][kMlpHid];
    for (int e = threadIdx.x; e < kMlpParams; e += 256) {
        const float x = theta[e];
        w[e] = (bf16 && e >= kMlpOffW1) ? round_bf16(x) : x;
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int s = blockIdx.x * 8 + warp;
    if (s >= n) return;
    for (int i = lane; i < kMlpIn; i += 32) {
        const float z = (F[(int64_t)s * kMlpIn + i] - w[i]) / w[kMlpIn + i];
        z0[warp][i] = bf16 ? round_bf16(z) : z;
    }
    __syncwarp();
    for (int h = lane; h < kMlpHid; h += 32) {
        float a = w[kMlpOffB1 + h];
        for (int i = 0; i < kMlpIn; ++i) a = fmaf(z0[warp][i], w[kMlpOffW1 + i * kMlpHid + h], a);
        const float t = tanhf(a);
        h1[warp][h] = bf16 ? round_bf16(t) : t;
    }
    __syncwarp();
    for (int h = lane; h < kMlpHid; h += 32) {
        float a = w[kMlpOffB2 + h];
        for (int k = 0; k < kMlpHid; ++k) a = fmaf(h1[warp][k], w[kMlpOffW2 + k * kMlpHid + h], a);
        const float t = tanhf(a);
        h2[warp][h] = bf16 ? round_bf16(t) : t;
    }
    __syncwarp();
#pragma unroll
    for (int o = 0; o < kMlpOut; ++o) {
        float a = 0.f;
        for (int h = lane; h < kMlpHid; h += 32) a = fmaf(h2[warp][h], w[kMlpOffW3 + h * kMlpOut + o], a);
        a = warp_sum(a);
        if (lane == 0) {
            const float sv = a + w[kMlpOffB3 + o];
            out[(int64_t)s * kMlpOut + o] = sv * w[2 * kMlpIn + kMlpOut + o] + w[2 * kMlpIn + o];
        }
    }
}

__global__ void mlp_init_kernel(float* theta, uint64_t seed) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e < kMlpOffW1 || e >= kMlpParams) return;
    double a = 0.0;
    if (e < kMlpOffB1) a = sqrt(6.0 / (kMlpIn + kMlpHid));
    else if (e >= kMlpOffW2 && e < kMlpOffB2) a = sqrt(6.0 / (kMlpHid + kMlpHid));
    else if (e >= kMlpOffW3 && e < kMlpOffB3) a = sqrt(6.0 / (kMlpHid + kMlpOut));
    theta[e] = (float)(a * (2.0 * mlp_uniform(seed, (uint64_t)e) - 1.0));
}

__device__ __forceinline__ double block_sum256(double v, double* red) {
    v = warp_sum(v);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double r = 0.0;
    for (int k = 0; k < 8; ++k) r += red[k];
    return r;
}

// Block c: mean and population standard deviation of column c of [F | Y].
__global__ void __launch_bounds__(256) mlp_normaliser_kernel(const float* F, const float* Y, int n, float* theta) {
    __shared__ double red[8];
    const int c = blockIdx.x;
    const bool feat = c < kMlpIn;
    const float* src = feat ? F + c : Y + (c - kMlpIn);
    const int stride = feat ? kMlpIn : kMlpOut;
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) s += (double)src[(int64_t)i * stride];
    const double mean = block_sum256(s, red) / (double)n;
    double q = 0.0;
    for (int i = threadIdx.x; i < n; i += 256) {
        const double dv = (double)src[(int64_t)i * stride] - mean;
        q += dv * dv;
    }
    double sd = sqrt(block_sum256(q, red) / (double)n);
    if (!(sd > 0.0)) sd = 1.0;
    if (threadIdx.x == 0) {
        if (feat) {
            theta[c] = (float)mean;
            theta[kMlpIn + c] = (float)sd;
        } else {
            theta[2 * kMlpIn + (c - kMlpIn)] = (float)mean;
            theta[2 * kMlpIn + kMlpOut + (c - kMlpIn)] = (float)sd;
        }
    }
}

// Block p: the input vector of problem p (two-pass FP64 mean and variance).
__global__ void __launch_bounds__(256) mlp_features_kernel(const ciq_problem* probs, float* F) {
    __shared__ double red[8];
    __shared__ double mean[CIQ_MAX_DIM];
    const ciq_problem pr = probs[blockIdx.x];
    float* f = F + (int64_t)blockIdx.x * kMlpIn;
    const int d = pr.d;
    for (int k = 0; k < CIQ_MAX_DIM; ++k) {
        double s = 0.0;
        if (k < d)
            for (int64_t i = threadIdx.x; i < pr.N; i += 256) s += (double)pr.X[i * d + k];
        const double m = block_sum256(s, red) / (double)pr.N;
        if (threadIdx.x == 0) mean[k] = k < d ? m : 0.0;
    }
    __syncthreads();
    for (int k = 0; k < CIQ_MAX_DIM; ++k) {
        double q = 0.0;
        if (k < d)
            for (int64_t i = threadIdx.x; i < pr.N; i += 256) {
                const double dv = (double)pr.X[i * d + k] - mean[k];
                q += dv * dv;
            }
        const double var = block_sum256(q, red) / (double)pr.N;
        if (threadIdx.x == 0) {
            f[6 + k] = (float)mean[k];
            f[6 + CIQ_MAX_DIM + k] = k < d ? (float)var : 0.f;
        }
    }
    if (threadIdx.x == 0) {
        f[0] = (float)log((double)pr.N);
        f[1] = (float)d;
        f[2] = pr.kern.type == CIQ_RBF ? 0.f : 1.f;
        f[3] = (float)log(pr.kern.lengthscale);
        f[4] = (float)log(pr.kern.outputscale);
        f[5] = (float)log(fmax(pr.kern.noise, 1e-12));
    }
}

}  // namespace

cudaError_t launch_mlp_features(const ciq_problem* probs_dev, int P, float* F, cudaStream_t st) {
    mlp_features_kernel<<<P, 256, 0, st>>>(probs_dev, F);
    return cudaGetLastError();
}

cudaError_t launch_mlp_normaliser(const float* F, const float* Y, int n, float* theta, cudaStream_t st) {
    mlp_normaliser_kernel<<<kMlpIn + kMlpOut, 256, 0, st>>>(F, Y, n, theta);
    return cudaGetLastError();
}

cudaError_t launch_mlp_init(float* theta, uint64_t seed, cudaStream_t st) {
    mlp_init_kernel<<<(kMlpParams + 255) / 256, 256, 0, st>>>(theta, seed);
    return cudaGetLastError();
}

cudaError_t launch_mlp_loss_grad(const float* theta, const float* F, const float* Y, int n, double* loss,
                                 double* grad, cudaStream_t st) {
    const size_t sm = grad_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(mlp_grad_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(loss, 0, sizeof(double), st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(grad, 0, sizeof(double) * kMlpParams, st)) != cudaSuccess) return e;
    mlp_grad_kernel<<<(n + kCB - 1) / kCB, 256, sm, st>>>(theta, F, Y, n, loss, grad);
    return cudaGetLastError();
}

cudaError_t launch_mlp_train(float* theta, float* adam, const float* F, const float* Y, int n, int steps, int batch,
                             float lr, uint64_t seed, int first_step, float* losses, cudaStream_t st) {
    const size_t sm = train_smem_bytes();
    cudaError_t e = cudaFuncSetAttribute(mlp_train_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    mlp_train_kernel<<<1, 256, sm, st>>>(theta, adam, adam + kMlpParams, F, Y, n, steps, batch, lr, seed, first_step,
                                         losses);
    return cudaGetLastError();
}

cudaError_t launch_mlp_predict(const float* theta, const float* F, int n, float* out, int bf16, cudaStream_t st) {
    mlp_predict_kernel<<<(n + 7) / 8, 256, 0, st>>>(theta, F, n, out, bf16);
    return cudaGetLastError();
}

}  // namespace ciq
