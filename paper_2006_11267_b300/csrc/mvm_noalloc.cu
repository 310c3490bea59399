// Allocation-free variant of the kernel MVM (ciq_kernel_mvm_noalloc).
//
// Some callers cannot call cudaMalloc: code whose device memory is owned by
// another allocator (a framework's caching allocator, a memory pool handed to
// a plugin), and latency-critical loops where an allocation, with the device
// synchronisation that cudaMalloc/cudaFree can imply, is not allowed.  This
// entry point takes its scratch (the points divided by the lengthscale and a
// zero-padded copy of V) from one file-scope device array of fixed size, so
// a call allocates nothing.  The array exists once per GPU that loads the
// library and stays until the process exits.
#include <mutex>

#include "host_checks.cuh"
#include "kernels.cuh"

namespace {

using namespace ciq;

// 16 MiB of scratch: Npad * dp + T * Npad floats must fit (for example
// N = 50,000, d = 6, T = 64 needs 3.6 M floats).
constexpr size_t kNoAllocScratchFloats = size_t(4) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kNoAllocScratchFloats];

std::mutex g_scratch_mu;
float* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device.  In host code
// the symbol g_noalloc_scratch names a host-side stand-in, not device memory,
// so the address is looked up once per device with that device current and
// kept for the life of the process.  The cache does not survive a reset of
// the device's primary context (cudaDeviceReset): the module is loaded again
// after one and the array may move, so a process that resets a device must
// not call this entry point on it afterwards.
cudaError_t scratch_on_current_device(float** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<float*>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" size_t ciq_noalloc_scratch_floats(void) { return kNoAllocScratchFloats; }

extern "C" ciq_status ciq_kernel_mvm_noalloc(const float* X, int64_t N, int d, const ciq_kernel* kern,
                                             const float* V, int T, float* out, ciq_stream_t stream) {
    if (!X || !V || !out || N < 1 || d < 1 || d > CIQ_MAX_DIM || T < 1 || !valid_kernel(kern))
        return CIQ_ERR_ARG;
    const int64_t Npad = round_up(N, kRowPad);
    const int dp = dim_pad(d);
    const int64_t x_floats = round_up(Npad * dp, 64);
    const double need = (double)x_floats + (double)T * (double)Npad;
    if (need > (double)kNoAllocScratchFloats) return CIQ_ERR_SCRATCH_TOO_SMALL;
    if (!device_accessible(X) || !device_accessible(V) || !device_accessible(out)) return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    float* scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    float* Xp = scratch;
    float* Vp = scratch + x_floats;
    if (e == cudaSuccess) e = launch_prepare_points<float, float>(X, N, d, Npad, dp, 1.0 / kern->lengthscale, Xp, st);
    // The scratch keeps the previous call's contents: the padded rows of V
    // must read as zero, so the whole V region is cleared first.
    if (e == cudaSuccess) e = cudaMemsetAsync(Vp, 0, sizeof(float) * (size_t)T * Npad, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Vp, sizeof(float) * Npad, V, sizeof(float) * N, sizeof(float) * N, T,
                              cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        MvmArgs<float> a{};
        a.X = Xp;
        a.N = N;
        a.Npad = Npad;
        a.dp = dp;
        a.kt = kern->type;
        a.s = (float)kern->outputscale;
        a.noise = (float)kern->noise;
        a.V = Vp;
        a.ldv = Npad;
        a.T = T;
        a.mode = kPlain;
        a.out = out;
        a.ldo = N;
        e = launch_mvm_simt(a, st);
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CIQ_ERR_NOMEM : CIQ_ERR_CUDA;
    }
    return CIQ_OK;
}
