// Shared device helpers of libciq (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ciq.h"

#define CIQ_HD __host__ __device__ __forceinline__

namespace ciq {

// Row padding of every workspace vector: all N-vectors are stored with a
// leading dimension that is a multiple of this, and the padded rows hold 0.
constexpr int kRowPad = 128;
constexpr int kMaxDimPad = 16;   // CIQ_MAX_DIM rounded to a multiple of 4

constexpr double kLog2e = 1.4426950408889634;
constexpr double kSqrt5 = 2.2360679774997896;

CIQ_HD int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

// exp2 on the SFU (PTX ex2.approx.ftz.f32; relative error about 2^-22).
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// sqrt on the SFU (PTX sqrt.approx.ftz.f32).
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Kernel value from the squared distance of points already divided by the
// lengthscale (r2 = ||x - x'||^2 / l^2), times the outputscale s.
//   RBF:        s exp(-r2 / 2)
//   Matern-5/2: s (1 + a + a^2/3) exp(-a),  a = sqrt(5 r2)
// FAST selects the SFU approximations (ex2.approx, sqrt.approx) used by the
// tensor-core tiles; otherwise CUDA's accurate expf/sqrtf (the plain FP32 path).
template <int KT, bool FAST = false>
__device__ __forceinline__ float kernel_value(float r2, float s) {
    if (KT == CIQ_RBF) {
        if (FAST) return s * ex2_approx(r2 * (float)(-0.5 * kLog2e));
        return s * expf(-0.5f * r2);
    } else {
        const float a = FAST ? sqrt_approx(r2 * 5.0f) : sqrtf(r2 * 5.0f);
        const float e = FAST ? ex2_approx(a * (float)(-kLog2e)) : expf(-a);
        return s * fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f) * e;
    }
}

template <int KT, bool FAST = false>
__device__ __forceinline__ double kernel_value(double r2, double s) {
    if (KT == CIQ_RBF) {
        return s * exp(-0.5 * r2);
    } else {
        double a = sqrt(5.0 * r2);
        return s * (1.0 + a + a * a / 3.0) * exp(-a);
    }
}

// (hi, lo) += x with Knuth's 2Sum: hi + lo carries the sum to about twice
// the working precision.
template <typename T>
__device__ __forceinline__ void two_sum_into(T& hi, T& lo, T x) {
    const T s = hi + x;
    const T bp = s - hi;
    const T err = (hi - (s - bp)) + (x - bp);
    hi = s;
    lo += err;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

}  // namespace ciq
