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

namespace ciq {

namespace {

template <typename R, int KT, int TC, int DP>
__global__ void __launch_bounds__(256) mvm_narrow(MvmArgs<R> a) {
    if (a.stop && *a.stop) return;
    constexpr int BM = 32, BN = 256;
    __shared__ R sX[DP][BN];
    __shared__ R sV[BN][TC];
    __shared__ R red[8][BM][TC];
    __shared__ R redlo[8][BM][TC];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * BM;
    const int c0 = blockIdx.y * TC;
    R xi[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) xi[k] = a.X[(i0 + lane) * DP + k];
    // Per-tile partial sums, carried into a (hi, lo) pair by 2Sum after every
    // tile: the rounding error of the N-term sum stays at the tile level.
    R hi[TC], lo[TC];
#pragma unroll
    for (int c = 0; c < TC; ++c) { hi[c] = (R)0; lo[c] = (R)0; }
    const R s = a.s;
    for (int64_t j0 = 0; j0 < a.Npad; j0 += BN) {
        R acc[TC];
#pragma unroll
        for (int c = 0; c < TC; ++c) acc[c] = (R)0;
        __syncthreads();
        const int64_t j = j0 + tid;
        const bool in = j < a.Npad;
#pragma unroll
        for (int k = 0; k < DP; ++k) sX[k][tid] = in ? a.X[j * DP + k] : (R)0;
#pragma unroll
        for (int c = 0; c < TC; ++c)
            sV[tid][c] = (in && c0 + c < a.T) ? a.V[(int64_t)(c0 + c) * a.ldv + j] : (R)0;
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < 32; ++jj) {
            const int jl = warp * 32 + jj;
            R r2 = (R)0;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                R df = xi[k] - sX[k][jl];
                r2 = fma(df, df, r2);
            }
            const R kv = kernel_value<KT>(r2, s);
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[c] = fma(kv, sV[jl][c], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < TC; ++c) two_sum_into(hi[c], lo[c], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < TC; ++c) {
        red[warp][lane][c] = hi[c];
        redlo[warp][lane][c] = lo[c];
    }
    __syncthreads();
    if (warp != 0) return;
    const int64_t i = i0 + lane;
#pragma unroll
    for (int c = 0; c < TC; ++c) {
        const int col = c0 + c;
        if (col >= a.T) break;
        double od = 0.0;
#pragma unroll
        for (int w = 0; w < 8; ++w) od += (double)red[w][lane][c] + (double)redlo[w][lane][c];
        const R o = (R)od;
        double qp = 0, pp = 0, qq = 0;
        lanczos_epilogue_value(a, i, col, o, qp, pp, qq);
        if (a.mode == kLanczos) {
            qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
            if (lane == 0) {
                double* dst = a.partials + ((int64_t)blockIdx.x * a.T + col) * 3;
                dst[0] = qp; dst[1] = pp; dst[2] = qq;
            }
        }
    }
}

template <int KT, int TC, int DP>
__global__ void __launch_bounds__(256) mvm_wide(MvmArgs<float> a) {
    if (a.stop && *a.stop) return;
    constexpr int BM = 64, BN = 64, MR = 4, MC = TC / 16;
    constexpr int LDP = BM + 4, LDV = TC + 4, LDO = TC + 1;
    static_assert(BN * LDP >= BM * LDO, "output tile must fit in the P buffer");
    __shared__ __align__(16) float sXj[DP][BN];
    __shared__ __align__(16) float sP[BN * LDP];
    __shared__ __align__(16) float sV[BN * LDV];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * BM;
    const int c0 = blockIdx.y * TC;
    const int pi = tid & 63, pj0 = (tid >> 6) * 16;
    const int ty = tid >> 4, tx = tid & 15;
    float xi[DP];
#pragma unroll
    for (int k = 0; k < DP; ++k) xi[k] = a.X[(i0 + pi) * DP + k];
    // Per-tile partial sums carried into (hi, lo) pairs by 2Sum (see mvm_narrow).
    float hi[MR][MC], lo[MR][MC];
#pragma unroll
    for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) { hi[r][c] = 0.f; lo[r][c] = 0.f; }
    const float s = a.s;
    for (int64_t j0 = 0; j0 < a.Npad; j0 += BN) {
        float acc[MR][MC];
#pragma unroll
        for (int r = 0; r < MR; ++r)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[r][c] = 0.f;
        __syncthreads();
        for (int e = tid; e < DP * BN; e += 256) sXj[e % DP][e / DP] = a.X[j0 * DP + e];
        for (int e = tid; e < BN * TC; e += 256) {
            const int c = e / BN, j = e % BN;
            sV[j * LDV + c] = (c0 + c < a.T) ? a.V[(int64_t)(c0 + c) * a.ldv + j0 + j] : 0.f;
        }
        __syncthreads();
#pragma unroll 4
        for (int jj = 0; jj < 16; ++jj) {
            const int j = pj0 + jj;
            float r2 = 0.f;
#pragma unroll
            for (int k = 0; k < DP; ++k) {
                float df = xi[k] - sXj[k][j];
                r2 = fmaf(df, df, r2);
            }
            sP[j * LDP + pi] = kernel_value<KT>(r2, s);
        }
        __syncthreads();
#pragma unroll 8
        for (int j = 0; j < BN; ++j) {
            const float4 pa = *reinterpret_cast<const float4*>(&sP[j * LDP + ty * MR]);
            float bv[MC];
#pragma unroll
            for (int c = 0; c < MC; c += 4) {
                const float4 t4 = *reinterpret_cast<const float4*>(&sV[j * LDV + tx * MC + c]);
                bv[c] = t4.x; bv[c + 1] = t4.y; bv[c + 2] = t4.z; bv[c + 3] = t4.w;
            }
            const float av[4] = {pa.x, pa.y, pa.z, pa.w};
#pragma unroll
            for (int r = 0; r < MR; ++r)
#pragma unroll
                for (int c = 0; c < MC; ++c) acc[r][c] = fmaf(av[r], bv[c], acc[r][c]);
        }
#pragma unroll
        for (int r = 0; r < MR; ++r)
#pragma unroll
            for (int c = 0; c < MC; ++c) two_sum_into(hi[r][c], lo[r][c], acc[r][c]);
    }
    __syncthreads();
    float* sO = sP;
#pragma unroll
    for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) sO[(ty * MR + r) * LDO + tx * MC + c] = hi[r][c] + lo[r][c];
    __syncthreads();
    constexpr int TPC = 256 / TC;          // threads per column
    constexpr int RPT = BM / TPC;          // rows per thread
    const int col_l = tid / TPC, part = tid % TPC;
    const int col = c0 + col_l;
    double qp = 0, pp = 0, qq = 0;
    if (col < a.T) {
        for (int rr = 0; rr < RPT; ++rr) {
            const int r = part * RPT + rr;
            lanczos_epilogue_value(a, i0 + r, col, sO[r * LDO + col_l], qp, pp, qq);
        }
    }
    if (a.mode == kLanczos) {
#pragma unroll
        for (int o = 1; o < TPC; o <<= 1) {
            qp += __shfl_xor_sync(0xffffffffu, qp, o);
            pp += __shfl_xor_sync(0xffffffffu, pp, o);
            qq += __shfl_xor_sync(0xffffffffu, qq, o);
        }
        if (part == 0 && col < a.T) {
            double* dst = a.partials + ((int64_t)blockIdx.x * a.T + col) * 3;
            dst[0] = qp; dst[1] = pp; dst[2] = qq;
        }
    }
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
