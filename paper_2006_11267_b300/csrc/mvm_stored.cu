// Stored-K variant of the kernel MVM: K = K_XX + sigma^2 I formed once in
// device memory (FP32, row-major, leading dimension ldk), then streamed by
// every msMINRES iteration (the O(J N^2) runtime of Sec. 3.3 for an explicit
// matrix).  Padded rows and columns of the stored matrix hold 0.
//
//  * kernel_matrix_kernel: 64 x 64 tiles of K from the points (accurate expf).
//  * stored_wide (T >= 17): 64 x 64 tile of K loaded with float4 reads into
//    shared memory, register-tiled 64 x 64 x TC product with V, compensated
//    accumulation over tiles, Lanczos epilogue (same as the on-the-fly MVM).
//  * stored_narrow (T <= 16, column groups of up to 8): a warp takes 1, 2 or
//    4 rows with float4 reads along them, each V float4 from L2 shared by the
//    warp's rows; HBM-bound.
#include <type_traits>

#include "kernels.cuh"
#include "mvm_stored.cuh"

namespace ciq {

namespace {

template <int KT, int DP>
__global__ void __launch_bounds__(256) kernel_matrix_kernel(const float* Xp, int64_t N, int64_t Npad,
                                                            float s, float noise, float* Kmat, int64_t ldk,
                                                            int64_t ncols) {
    __shared__ float sXi[64][DP + 1];
    __shared__ float sXj[64][DP + 1];
    const int64_t i0 = (int64_t)blockIdx.y * 64, j0 = (int64_t)blockIdx.x * 64;
    const int tid = threadIdx.x;
    for (int e = tid; e < 64 * DP; e += 256) {
        sXi[e / DP][e % DP] = Xp[(i0 + e / DP) * DP + e % DP];
        sXj[e / DP][e % DP] = Xp[(j0 + e / DP) * DP + e % DP];
    }
    __syncthreads();
    const int jl = tid & 63;
    const int64_t j = j0 + jl;
    for (int il = tid >> 6; il < 64; il += 4) {
        const int64_t i = i0 + il;
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < DP; ++k) {
            const float df = sXi[il][k] - sXj[jl][k];
            r2 = fmaf(df, df, r2);
        }
        float v = 0.f;
        if (i < N && j < N) v = kernel_value<KT>(r2, s) + (i == j ? noise : 0.f);
        if (j < ncols) Kmat[i * ldk + j] = v;
    }
}

template <int TC>
__global__ void __launch_bounds__(256) stored_wide(const float* Kmat, int64_t ldk, MvmArgs<float> a) {
    if (a.stop && *a.stop) return;
    constexpr int BM = 64, BN = 64, MR = 4, MC = TC / 16;
    constexpr int LDP = BM + 4, LDV = TC + 4, LDO = TC + 1;
    __shared__ __align__(16) float sP[BN * LDP];
    __shared__ __align__(16) float sV[BN * LDV];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.x * BM;
    const int c0 = blockIdx.y * TC;
    const int ty = tid >> 4, tx = tid & 15;
    float hi[MR][MC], lo[MR][MC];
#pragma unroll
    for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) { hi[r][c] = 0.f; lo[r][c] = 0.f; }
    for (int64_t j0 = 0; j0 < a.Npad; j0 += BN) {
        float acc[MR][MC];
#pragma unroll
        for (int r = 0; r < MR; ++r)
#pragma unroll
            for (int c = 0; c < MC; ++c) acc[r][c] = 0.f;
        __syncthreads();
        // K tile: 64 rows x 64 floats = 1024 float4, 4 per thread, stored transposed.
        for (int e = tid; e < BM * (BN / 4); e += 256) {
            const int il = e / (BN / 4), jq = e % (BN / 4);
            const float4 k4 = *reinterpret_cast<const float4*>(Kmat + (i0 + il) * ldk + j0 + 4 * jq);
            sP[(4 * jq + 0) * LDP + il] = k4.x;
            sP[(4 * jq + 1) * LDP + il] = k4.y;
            sP[(4 * jq + 2) * LDP + il] = k4.z;
            sP[(4 * jq + 3) * LDP + il] = k4.w;
        }
        for (int e = tid; e < BN * TC; e += 256) {
            const int c = e / BN, j = e % BN;
            sV[j * LDV + c] = (c0 + c < a.T) ? a.V[(int64_t)(c0 + c) * a.ldv + j0 + j] : 0.f;
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
    constexpr int TPC = 256 / TC;
    constexpr int RPT = BM / TPC;
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

// R rows per warp, 8 warps per block; TC columns of V per launch column
// group.  Each float4 of V feeds the warp's R rows, so V is read from L2 TC / R
// times per float4 of K (R = TC / 2, at least 1), which keeps the kernel on
// the HBM stream of K.  Per (row, column) the sum order is the same for any R.
template <int TC, int R>
__global__ void __launch_bounds__(256) stored_narrow(const float* Kmat, int64_t ldk, MvmArgs<float> a) {
    if (a.stop && *a.stop) return;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t i0 = ((int64_t)blockIdx.x * 8 + warp) * R;
    const int c0 = blockIdx.y * TC;
    float hi[R][TC], lo[R][TC];
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int c = 0; c < TC; ++c) { hi[r][c] = 0.f; lo[r][c] = 0.f; }
    for (int64_t j0 = 0; j0 < a.Npad; j0 += 1024) {
        float acc[R][TC];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) acc[r][c] = 0.f;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t j = j0 + q * 128 + lane * 4;
            if (j < a.Npad) {
                float4 v4[TC];
#pragma unroll
                for (int c = 0; c < TC; ++c)
                    v4[c] = c0 + c < a.T ? *reinterpret_cast<const float4*>(a.V + (int64_t)(c0 + c) * a.ldv + j)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float4 k4 = *reinterpret_cast<const float4*>(Kmat + (i0 + r) * ldk + j);
#pragma unroll
                    for (int c = 0; c < TC; ++c)
                        acc[r][c] = fmaf(k4.x, v4[c].x, fmaf(k4.y, v4[c].y, fmaf(k4.z, v4[c].z, fmaf(k4.w, v4[c].w, acc[r][c]))));
                }
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int c = 0; c < TC; ++c) two_sum_into(hi[r][c], lo[r][c], acc[r][c]);
    }
    __shared__ double red[8][TC][3];
#pragma unroll
    for (int c = 0; c < TC; ++c) {
        const int col = c0 + c;
        double qp = 0, pp = 0, qq = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double o = warp_sum((double)hi[r][c] + (double)lo[r][c]);
            if (lane == 0 && col < a.T) lanczos_epilogue_value(a, i0 + r, col, (float)o, qp, pp, qq);
        }
        if (lane == 0) { red[warp][c][0] = qp; red[warp][c][1] = pp; red[warp][c][2] = qq; }
    }
    if (a.mode != kLanczos) return;
    __syncthreads();
    if (threadIdx.x < TC * 3) {
        const int c = threadIdx.x / 3, k = threadIdx.x % 3;
        if (c0 + c < a.T) {
            double sum = 0.0;
            for (int w = 0; w < 8; ++w) sum += red[w][c][k];
            a.partials[((int64_t)blockIdx.x * a.T + c0 + c) * 3 + k] = sum;
        }
    }
}

template <int KT>
cudaError_t km_dp(const float* Xp, int64_t N, int64_t Npad, int dp, float s, float noise, float* Kmat,
                  int64_t ldk, int64_t ncols, cudaStream_t st) {
    dim3 grid((unsigned)((ncols + 63) / 64), (unsigned)(Npad / 64));
    switch (dp) {
        case 4: kernel_matrix_kernel<KT, 4><<<grid, 256, 0, st>>>(Xp, N, Npad, s, noise, Kmat, ldk, ncols); break;
        case 8: kernel_matrix_kernel<KT, 8><<<grid, 256, 0, st>>>(Xp, N, Npad, s, noise, Kmat, ldk, ncols); break;
        case 12: kernel_matrix_kernel<KT, 12><<<grid, 256, 0, st>>>(Xp, N, Npad, s, noise, Kmat, ldk, ncols); break;
        case 16: kernel_matrix_kernel<KT, 16><<<grid, 256, 0, st>>>(Xp, N, Npad, s, noise, Kmat, ldk, ncols); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace

// Column group of the narrow kernel for T <= 16 columns and its rows per warp.
static int narrow_tc(int T) { return T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : 8; }
static int narrow_rows(int T) { return narrow_tc(T) <= 2 ? 1 : narrow_tc(T) / 2; }

int64_t stored_row_tiles(int64_t Npad, int T) { return T >= 17 ? Npad / 64 : Npad / (8 * narrow_rows(T)); }

cudaError_t launch_kernel_matrix(const float* Xp, int64_t N, int64_t Npad, int dp, int kt, float s, float noise,
                                 float* Kmat, int64_t ldk, int64_t ncols, cudaStream_t st) {
    // ncols <= ldk columns are written per row (Npad for the solve's padded copy).
    if (Npad % 64 != 0 || ncols > ldk) return cudaErrorInvalidValue;
    return kt == CIQ_RBF ? km_dp<CIQ_RBF>(Xp, N, Npad, dp, s, noise, Kmat, ldk, ncols, st)
                         : km_dp<CIQ_MATERN52>(Xp, N, Npad, dp, s, noise, Kmat, ldk, ncols, st);
}

cudaError_t launch_stored_mvm(const float* Kmat, int64_t ldk, const MvmArgs<float>& args, cudaStream_t st) {
    if (args.Npad % 64 != 0 || ldk % 4 != 0 || ldk < args.Npad) return cudaErrorInvalidValue;
    MvmArgs<float> a = args;
    a.noise = 0.f;          // the stored matrix already holds sigma^2 on its diagonal
    if (a.T >= 17) {
        const int TC = a.T > 32 ? 64 : 32;
        dim3 grid((unsigned)(a.Npad / 64), (unsigned)((a.T + TC - 1) / TC));
        if (TC == 64) stored_wide<64><<<grid, 256, 0, st>>>(Kmat, ldk, a);
        else stored_wide<32><<<grid, 256, 0, st>>>(Kmat, ldk, a);
    } else {
        const int TC = narrow_tc(a.T);
        dim3 grid((unsigned)(a.Npad / (8 * narrow_rows(a.T))), (unsigned)((a.T + TC - 1) / TC));
        switch (TC) {
            case 1: stored_narrow<1, 1><<<grid, 256, 0, st>>>(Kmat, ldk, a); break;
            case 2: stored_narrow<2, 1><<<grid, 256, 0, st>>>(Kmat, ldk, a); break;
            case 4: stored_narrow<4, 2><<<grid, 256, 0, st>>>(Kmat, ldk, a); break;
            default: stored_narrow<8, 4><<<grid, 256, 0, st>>>(Kmat, ldk, a); break;
        }
    }
    return cudaGetLastError();
}

}  // namespace ciq
