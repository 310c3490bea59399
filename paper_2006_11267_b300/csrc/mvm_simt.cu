// On-the-fly kernel MVM on CUDA cores (FP32 or FP64): O = (K_XX + sigma^2 I) V
// with K never stored (the "map-reduce" MVM of Sec. 3.3, Property 1).  This is
// the plain-precision path: distances from coordinate differences, kernel
// values on the SFU (FP32) or in IEEE FP64, products on FMA units.
//
//  * mvm_narrow (T <= 8 per launch column group): one row per lane, the 8
//    warps of a block split each 256-point tile of K's columns, partial sums
//    reduced through shared memory.
//  * mvm_wide (FP32, 17 <= T): 64 x 64 tile of K formed in shared memory,
//    then a register-tiled 64 x 64 x TC product with the V tile.
//
// Both end with the epilogue selected by MvmArgs::mode (kernels.cuh), which in
// kLanczos mode fuses the first half of a Lanczos step of Algorithm
// "msMINRES": p = K q_j - beta_j q_{j-1} and the FP64 partial sums of q.p,
// p.p and q.q for alpha_j and beta_{j+1}.
#include <type_traits>

#include "kernels.cuh"
#include "mvm_simt_body.cuh"

namespace ciq {

namespace {

template <typename R, int KT, int TC, int DP>
__global__ void __launch_bounds__(256) mvm_narrow(MvmArgs<R> a) {
    mvm_narrow_body<R, KT, TC, DP>(a, blockIdx.x, blockIdx.y);
}

template <int KT, int TC, int DP>
__global__ void __launch_bounds__(256) mvm_wide(MvmArgs<float> a) {
    mvm_wide_body<KT, TC, DP>(a, blockIdx.x, blockIdx.y);
}

template <typename R, typename Rin>
__global__ void prepare_points_kernel(const Rin* X, int64_t N, int d, int64_t Npad, int dp,
                                      double inv_ls, R* Xp) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= Npad * dp) return;
    const int64_t i = e / dp;
    const int k = (int)(e % dp);
    Xp[e] = (i < N && k < d) ? (R)((double)X[i * d + k] * inv_ls) : (R)0;
}

template <typename R>
bool use_wide(int T) { return std::is_same<R, float>::value && T >= 17; }

template <typename R, int KT, int TC>
cudaError_t narrow_dp(const MvmArgs<R>& a, dim3 grid, cudaStream_t st) {
    switch (a.dp) {
        case 4: mvm_narrow<R, KT, TC, 4><<<grid, 256, 0, st>>>(a); break;
        case 8: mvm_narrow<R, KT, TC, 8><<<grid, 256, 0, st>>>(a); break;
        case 12: mvm_narrow<R, KT, TC, 12><<<grid, 256, 0, st>>>(a); break;
        case 16: mvm_narrow<R, KT, TC, 16><<<grid, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KT, int TC>
cudaError_t wide_dp(const MvmArgs<float>& a, dim3 grid, cudaStream_t st) {
    switch (a.dp) {
        case 4: mvm_wide<KT, TC, 4><<<grid, 256, 0, st>>>(a); break;
        case 8: mvm_wide<KT, TC, 8><<<grid, 256, 0, st>>>(a); break;
        case 12: mvm_wide<KT, TC, 12><<<grid, 256, 0, st>>>(a); break;
        case 16: mvm_wide<KT, TC, 16><<<grid, 256, 0, st>>>(a); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <typename R, int KT>
cudaError_t launch_kt(const MvmArgs<R>& a, cudaStream_t st) {
    if constexpr (std::is_same<R, float>::value) {
        if (use_wide<R>(a.T)) {
            const int TC = a.T > 32 ? 64 : 32;
            dim3 grid((unsigned)(a.Npad / 64), (unsigned)((a.T + TC - 1) / TC));
            return TC == 64 ? wide_dp<KT, 64>(a, grid, st) : wide_dp<KT, 32>(a, grid, st);
        }
    }
    // FP64 column groups stay at <= 2 so the static shared memory fits in 48 KB.
    const int tc_max = std::is_same<R, float>::value ? 8 : 2;
    int TC = a.T <= 1 ? 1 : a.T <= 2 ? 2 : a.T <= 4 ? 4 : 8;
    if (TC > tc_max) TC = tc_max;
    dim3 grid((unsigned)(a.Npad / 32), (unsigned)((a.T + TC - 1) / TC));
    switch (TC) {
        case 1: return narrow_dp<R, KT, 1>(a, grid, st);
        case 2: return narrow_dp<R, KT, 2>(a, grid, st);
        default:
            if constexpr (std::is_same<R, float>::value) {
                return TC == 4 ? narrow_dp<R, KT, 4>(a, grid, st) : narrow_dp<R, KT, 8>(a, grid, st);
            }
            return cudaErrorInvalidValue;
    }
}

}  // namespace

template <typename R>
int64_t mvm_simt_row_tiles(int64_t Npad, int T) { return use_wide<R>(T) ? Npad / 64 : Npad / 32; }

template int64_t mvm_simt_row_tiles<float>(int64_t, int);
template int64_t mvm_simt_row_tiles<double>(int64_t, int);

template <typename R>
cudaError_t launch_mvm_simt(const MvmArgs<R>& a, cudaStream_t st) {
    if (a.Npad % kRowPad != 0 || a.T < 1) return cudaErrorInvalidValue;
    return a.kt == CIQ_RBF ? launch_kt<R, CIQ_RBF>(a, st) : launch_kt<R, CIQ_MATERN52>(a, st);
}

template cudaError_t launch_mvm_simt<float>(const MvmArgs<float>&, cudaStream_t);
template cudaError_t launch_mvm_simt<double>(const MvmArgs<double>&, cudaStream_t);

template <typename R, typename Rin>
cudaError_t launch_prepare_points(const Rin* X, int64_t N, int d, int64_t Npad, int dp,
                                  double inv_ls, R* Xp, cudaStream_t st) {
    const int64_t total = Npad * dp;
    prepare_points_kernel<R, Rin><<<(unsigned)((total + 255) / 256), 256, 0, st>>>(X, N, d, Npad, dp,
                                                                                     inv_ls, Xp);
    return cudaGetLastError();
}

template cudaError_t launch_prepare_points<float, float>(const float*, int64_t, int, int64_t, int,
                                                         double, float*, cudaStream_t);
template cudaError_t launch_prepare_points<double, double>(const double*, int64_t, int, int64_t,
                                                           int, double, double*, cudaStream_t);

}  // namespace ciq
