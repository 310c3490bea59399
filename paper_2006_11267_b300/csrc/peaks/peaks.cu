// Throughput microbenchmarks for the roofline denominators beyond the copy
// rate and the BF16 GEMM rate: SFU exp2 (ex2.approx.ftz.f32, the SFU op of
// every kernel entry), FP32 FMA and FP64 FMA.  Each thread runs 8 independent dependent
// chains; the grid is 8 CTAs of 256 threads per SM.  Built as its own library
// (libciq_peaks.so); the solver does not use it.
#include <cuda_runtime.h>
#include <stdint.h>

namespace {

__device__ __forceinline__ float ex2f(float x) {
    float y;
    asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// clk (optional): thread 0 of block 0 writes the SM clock count and the
// global timer (ns) at its start and end, so the run's own SM clock is known.
__global__ void ex2_kernel(float* out, int iters, unsigned long long* clk) {
    unsigned long long c0 = 0, t0 = 0;
    if (clk && blockIdx.x == 0 && threadIdx.x == 0) {
        c0 = clock64();
        t0 = globaltimer_ns();
    }
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = -1.0f - 1e-3f * (float)(threadIdx.x + k);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = -ex2f(a[k]);
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
    if (clk && blockIdx.x == 0 && threadIdx.x == 0) {
        clk[0] = clock64() - c0;
        clk[1] = globaltimer_ns() - t0;
    }
}

template <typename T>
__global__ void fma_kernel(T* out, int iters) {
    T a[8];
    const T b = (T)0.999999, c = (T)1e-7;
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (T)(threadIdx.x + k) * (T)1e-3;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename F>
int time_kernel(F launch, double* ms_out) {
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return 2;
    launch();                                   // warm-up
    cudaEventRecord(e0);
    launch();
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms_out = ms;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

}  // namespace

// ops/s of ex2.approx.ftz.f32 over the whole device.
extern "C" int ciq_peak_sfu_ex2(double* ops_per_s, double* ms) {
    const int blocks = 8 * sm_count(), threads = 256, iters = 4096;
    float* out = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 2;
    int rc = time_kernel([&] { ex2_kernel<<<blocks, threads>>>(out, iters, nullptr); }, ms);
    *ops_per_s = (double)blocks * threads * iters * 8 / (*ms * 1e-3);
    cudaFree(out);
    return rc;
}

// The same ex2 throughput over a longer run (about 20 ms), with the SM clock
// the run itself saw: ops/s, ex2 per SM per clock cycle, and SM MHz (clock64
// cycles over global-timer ns of one thread that lives for the whole launch).
extern "C" int ciq_peak_sfu_ex2_clock(double* ops_per_s, double* ms, double* per_sm_per_clk, double* sm_mhz) {
    const int sms = sm_count(), blocks = 8 * sms, threads = 256, iters = 65536;
    float* out = nullptr;
    unsigned long long* clk = nullptr;
    if (cudaMalloc(&out, sizeof(float) * blocks * threads) != cudaSuccess) return 2;
    if (cudaMalloc(&clk, 2 * sizeof(unsigned long long)) != cudaSuccess) { cudaFree(out); return 2; }
    int rc = time_kernel([&] { ex2_kernel<<<blocks, threads>>>(out, iters, clk); }, ms);
    unsigned long long h[2] = {0, 0};
    if (cudaMemcpy(h, clk, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) rc = 2;
    const double ops = (double)blocks * threads * iters * 8;
    *ops_per_s = ops / (*ms * 1e-3);
    *sm_mhz = h[1] ? (double)h[0] / (double)h[1] * 1e3 : 0.0;
    // Cycles of the whole launch at that clock.
    const double cycles = (*ms * 1e-3) * (*sm_mhz * 1e6);
    *per_sm_per_clk = cycles > 0 ? ops / (cycles * sms) : 0.0;
    cudaFree(out);
    cudaFree(clk);
    return rc;
}

// FLOP/s (2 per FMA) of FP32 or FP64 FMA over the whole device.
extern "C" int ciq_peak_fma(int fp64, double* flops, double* ms) {
    const int blocks = 8 * sm_count(), threads = 256, iters = fp64 ? 256 : 8192;
    void* out = nullptr;
    if (cudaMalloc(&out, 8 * (size_t)blocks * threads) != cudaSuccess) return 2;
    int rc;
    if (fp64)
        rc = time_kernel([&] { fma_kernel<double><<<blocks, threads>>>((double*)out, iters); }, ms);
    else
        rc = time_kernel([&] { fma_kernel<float><<<blocks, threads>>>((float*)out, iters); }, ms);
    *flops = 2.0 * blocks * threads * iters * 8 / (*ms * 1e-3);
    cudaFree(out);
    return rc;
}
