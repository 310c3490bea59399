// Bodies of the CUDA-core kernel MVMs (see mvm_simt.cu), written against
// explicit block coordinates so that the single-problem kernels and the
// batched kernels (batched.cu) run the same code.
#pragma once

#include "kernels.cuh"

namespace ciq {
namespace {

template <typename R, int KT, int TC, int DP>
__device__ __forceinline__ void mvm_narrow_body(const MvmArgs<R>& a, int bx, int by) {
    if (a.stop && *a.stop) return;
    constexpr int BM = 32, BN = 256;
    __shared__ R sX[DP][BN];
    __shared__ R sV[BN][TC];
    __shared__ R red[8][BM][TC];
    __shared__ R redlo[8][BM][TC];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)bx * BM;
    const int c0 = by * TC;
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
        lanczos_epilogue_value<R, true>(a, i, col, o, qp, pp, qq, (R)(od - (double)o));
        if (a.mode == kLanczos) {
            qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
            if (lane == 0) {
                double* dst = a.partials + ((int64_t)bx * a.T + col) * 3;
                dst[0] = qp; dst[1] = pp; dst[2] = qq;
            }
        }
    }
}

template <int KT, int TC, int DP>
__device__ __forceinline__ void mvm_wide_body(const MvmArgs<float>& a, int bx, int by) {
    if (a.stop && *a.stop) return;
    constexpr int BM = 64, BN = 64, MR = 4, MC = TC / 16;
    constexpr int LDP = BM + 4, LDV = TC + 4, LDO = TC + 1;
    static_assert(BN * LDP >= BM * LDO, "output tile must fit in the P buffer");
    __shared__ __align__(16) float sXj[DP][BN];
    __shared__ __align__(16) float sP[BN * LDP];
    __shared__ __align__(16) float sV[BN * LDV];
    const int tid = threadIdx.x;
    const int64_t i0 = (int64_t)bx * BM;
    const int c0 = by * TC;
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
    // The output tile as a (leading, trailing) pair: leading parts over the
    // P buffer, trailing parts over the V buffer (both free now).
    float* sO = sP;
    float* sOlo = sV;
    static_assert(BN * LDV >= BM * LDO, "trailing parts must fit in the V buffer");
#pragma unroll
    for (int r = 0; r < MR; ++r)
#pragma unroll
        for (int c = 0; c < MC; ++c) {
            const float sum = hi[r][c] + lo[r][c];
            sO[(ty * MR + r) * LDO + tx * MC + c] = sum;
            sOlo[(ty * MR + r) * LDO + tx * MC + c] = (hi[r][c] - sum) + lo[r][c];
        }
    __syncthreads();
    constexpr int TPC = 256 / TC;          // threads per column
    constexpr int RPT = BM / TPC;          // rows per thread
    const int col_l = tid / TPC, part = tid % TPC;
    const int col = c0 + col_l;
    double qp = 0, pp = 0, qq = 0;
    if (col < a.T) {
        for (int rr = 0; rr < RPT; ++rr) {
            const int r = part * RPT + rr;
            lanczos_epilogue_value<float, true>(a, i0 + r, col, sO[r * LDO + col_l], qp, pp, qq, sOlo[r * LDO + col_l]);
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
            double* dst = a.partials + ((int64_t)bx * a.T + col) * 3;
            dst[0] = qp; dst[1] = pp; dst[2] = qq;
        }
    }
}

}  // namespace
}  // namespace ciq
