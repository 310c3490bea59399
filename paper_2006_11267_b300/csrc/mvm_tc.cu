// On-the-fly kernel MVM on the tcgen05 tensor cores (sm_103a).
//
// O = (K_XX + sigma^2 I) V without storing K (the map-reduce MVM of Sec. 3.3).
// One CTA owns 128 rows of K and streams the points and V in steps of 128
// columns (two 64-row operand tiles):
//
//   S   = U_i V_j^T on tensor cores, kind::f16, accumulator in TMEM.  Rows are
//         augmented, u = [c(x - m), -c^2 |x - m|^2 / 2, 1] and v = [c(x - m), 1,
//         -c^2 |x - m|^2 / 2], so S = -c^2 r^2 / 2 directly (norm expansion of
//         the distance; m is the centre of the points).  Each operand is split
//         into a 16-bit leading part and a 16-bit trailing part and S =
//         U_h V_h + U_h V_l + U_l V_h (three K-chunks of one MMA sequence):
//         about 22 significant bits with FP16 parts.  For d <= 6 the 8
//         augmented features fill half a chunk: two MMAs; with BF16 parts the
//         free half of the last chunk carries U_l V_l, so S has all four
//         products.
//   P   = k(r) / s from S on the SFU (RBF: ex2(S) with c^2 = log2 e; Matern-5/2:
//         a = sqrt(-10 S), (1 + a + a^2/3) ex2(-a log2 e)), split again into
//         leading/trailing 16-bit parts and written back over S in tensor
//         memory (tcgen05.st), so the product reads its A operand from TMEM
//         and shared-memory bandwidth is left to the B operands and copies.
//   O  += P_h Vt_h + P_h Vt_l + P_l Vt_h on tensor cores, accumulator in TMEM,
//         with Vt = V times a power of two per column, split like U.
//
// The operands are pre-arranged in global memory in the shared-memory layout
// of the MMA, so every step's tile is one bulk copy (cp.async.bulk)
// completing on an mbarrier, in three-stage rings.  Each CTA writes its
// column sums (a contiguous range of K's columns of one row tile); the
// finish kernel adds a tile's partial sums in split order and applies the
// same plain or Lanczos epilogue as the CUDA-core MVM.  Every wait is
// bounded: on timeout the CTA records an error flag, stops issuing, waits
// (bounded) for its own copies and MMAs in flight and frees its TMEM.
#include <algorithm>
#include <atomic>

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "batched.cuh"
#include "mvm_tc.cuh"
#include "tc_ptx.cuh"

namespace ciq {

namespace {

constexpr long long kWaitLimit = 4000000000LL;   // clock cycles, ~2 s at 2 GHz
constexpr int kUBytes = kTcBM * kTcRowBytes;      // 12 KiB
constexpr int kXBytes = kTcBN * kTcRowBytes;      // 6 KiB

template <bool HALF>
__device__ __forceinline__ uint16_t to16(float x) {
    if (HALF) return __half_as_ushort(__float2half_rn(x));
    return __bfloat16_as_ushort(__float2bfloat16_rn(x));
}

template <bool HALF>
__device__ __forceinline__ float from16(uint16_t u) {
    if (HALF) return __half2float(__ushort_as_half(u));
    return __bfloat162float(__ushort_as_bfloat16(u));
}

__device__ __forceinline__ uint32_t pack2(uint16_t lo, uint16_t hi) {
    return (uint32_t)lo | ((uint32_t)hi << 16);
}

// Convert a pair to 16-bit leading parts (packed, a in the low half) and the
// trailing parts.  The remainder a - hi(a) is one mixed-precision FMA
// (hi(a) x -1 + a, 16-bit a and b operands, FP32 addend; PTX ISA 8.6), so
// the leading part is never widened back to FP32 by a separate conversion.
// The remainder is exact in FP32 (hi(a) is a rounded to 8 or 11 bits), so
// the result equals (a - float(hi(a))) rounded to 16 bits bit for bit.
template <bool HALF>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    float ra, rb;
    if (HALF) {
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
        asm("{\n\t.reg .b16 h0, h1, m;\n\t"
            "mov.b32 {h0, h1}, %2;\n\t"
            "mov.b16 m, 0xBC00;\n\t"            // -1.0 in FP16
            "fma.rn.f32.f16 %0, h0, m, %3;\n\t"
            "fma.rn.f32.f16 %1, h1, m, %4;\n\t}"
            : "=f"(ra), "=f"(rb)
            : "r"(hi), "f"(a), "f"(b));
        asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(rb), "f"(ra));
    } else {
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(hi) : "f"(b), "f"(a));
        asm("{\n\t.reg .b16 h0, h1, m;\n\t"
            "mov.b32 {h0, h1}, %2;\n\t"
            "mov.b16 m, 0xBF80;\n\t"            // -1.0 in BF16
            "fma.rn.f32.bf16 %0, h0, m, %3;\n\t"
            "fma.rn.f32.bf16 %1, h1, m, %4;\n\t}"
            : "=f"(ra), "=f"(rb)
            : "r"(hi), "f"(a), "f"(b));
        asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(lo) : "f"(rb), "f"(ra));
    }
}

// Round to TF32 (10 stored mantissa bits), to nearest with ties away from
// zero; the result is a float whose 13 low mantissa bits are zero.
__device__ __forceinline__ uint32_t to_tf32(float x) {
    uint32_t u;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(u) : "f"(x));
    return u;
}

// ---------------------------------------------------------- operand prep --
// Centre of the points, one block of 256 threads, in a fixed summation order
// (so the operands, and every result, are reproducible bit for bit).  Thread
// s sums rows s, s + 256, ... as a (leading, trailing) float pair (2Sum;
// FP64 adds run at a few per clock per SM on this part); the 256 pairs are
// then combined in a fixed tree and converted to FP64 once.
__device__ __forceinline__ void tc_mean_body(const float* Xp, int64_t N, int dp, double* mean) {
    __shared__ float red_h[8][kMaxDimPad], red_l[8][kMaxDimPad];
    float h[kMaxDimPad], l[kMaxDimPad];
#pragma unroll
    for (int k = 0; k < kMaxDimPad; ++k) { h[k] = 0.f; l[k] = 0.f; }
    for (int64_t i = threadIdx.x; i < N; i += 256)
#pragma unroll
        for (int k = 0; k < kMaxDimPad; ++k)
            if (k < dp) two_sum_into(h[k], l[k], Xp[i * dp + k]);
#pragma unroll
    for (int k = 0; k < kMaxDimPad; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const float oh = __shfl_xor_sync(0xffffffffu, h[k], o);
            const float ol = __shfl_xor_sync(0xffffffffu, l[k], o);
            two_sum_into(h[k], l[k], oh);
            l[k] += ol;
        }
        if ((threadIdx.x & 31) == 0) {
            red_h[threadIdx.x >> 5][k] = h[k];
            red_l[threadIdx.x >> 5][k] = l[k];
        }
    }
    __syncthreads();
    if (threadIdx.x < kMaxDimPad) {
        const int k = threadIdx.x;
        float sh = 0.f, sl = 0.f;
        for (int w = 0; w < 8; ++w) {
            two_sum_into(sh, sl, red_h[w][k]);
            sl += red_l[w][k];
        }
        mean[k] = k < dp ? ((double)sh + (double)sl) / (double)N : 0.0;
    }
}

__global__ void __launch_bounds__(256) tc_mean_kernel(const float* Xp, int64_t N, int dp, double* mean) {
    tc_mean_body(Xp, N, dp, mean);
}

// One thread per row: u, v augmented and split, written in the operand layout
// [row/8][chunk 0..2][K-core 0..1][row%8][element%8] (16-bit elements).
template <bool HALF>
__device__ __forceinline__ void tc_points_body(const float* Xp, int64_t N, int64_t Npad, int dp, int d, float c,
                                               float c2half, const double* mean, uint8_t* ua, uint8_t* ub,
                                               int64_t row) {
    if (row >= Npad) return;
    float u[16], v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) { u[k] = 0.f; v[k] = 0.f; }
    if (row < N) {
        float n2 = 0.f;
        for (int k = 0; k < d; ++k) {
            const float xc = Xp[row * dp + k] - (float)mean[k];
            n2 = fmaf(xc, xc, n2);
            u[k] = c * xc;
            v[k] = c * xc;
        }
        u[d] = -c2half * n2;
        u[d + 1] = 1.f;
        v[d] = 1.f;
        v[d + 1] = -c2half * n2;
    }
    uint16_t uh[16], ul[16], vh[16], vl[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        uh[k] = to16<HALF>(u[k]);
        ul[k] = to16<HALF>(u[k] - from16<HALF>(uh[k]));
        vh[k] = to16<HALF>(v[k]);
        vl[k] = to16<HALF>(v[k] - from16<HALF>(vh[k]));
    }
    const uint16_t* achunk[3] = {uh, uh, ul};
    const uint16_t* bchunk[3] = {vh, vl, vh};
    // BF16 parts with at most 8 augmented features: only K-core 0 of each
    // chunk carries them, and K-core 1 of chunk 2 takes (u_l, v_l), so the
    // MMA over chunk 2 adds u_l v_l to u_l v_h and S has all four products of
    // the split (measured: 1.4e-4 against 2.4e-4 MVM error for Matern-5/2 at
    // lengthscale 0.1).  With FP16 parts the fourth product is below the
    // MVM's other errors (1.85e-6 either way at d = 6) and the 50,000-point
    // solve took 905 iterations with it against 897 without, so FP16 keeps
    // three.
    const bool narrow = !HALF && d + 2 <= 8;
    const size_t base = (size_t)(row >> 3) * kTcRowBytes * 8 + (size_t)(row & 7) * 16;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            const bool ll = narrow && ch == 2 && kc == 1;
            const uint16_t* a = ll ? ul : achunk[ch] + kc * 8;
            const uint16_t* b = ll ? vl : bchunk[ch] + kc * 8;
            const size_t off = base + (size_t)ch * 256 + (size_t)kc * 128;
            *reinterpret_cast<uint4*>(ua + off) =
                make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
            *reinterpret_cast<uint4*>(ub + off) =
                make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        }
    }
}

template <bool HALF>
__global__ void tc_points_kernel(const float* Xp, int64_t N, int64_t Npad, int dp, int d, float c,
                                 float c2half, const double* mean, uint8_t* ua, uint8_t* ub) {
    tc_points_body<HALF>(Xp, N, Npad, dp, d, c, c2half, mean, ua, ub, (int64_t)blockIdx.x * blockDim.x + threadIdx.x);
}

// Power-of-two scale per column so the scaled entries sit near 1.
__global__ void tc_vscale_kernel(const float* V, int64_t ldv, int64_t N, int T, int TP, float unit_scale,
                                 int unit, float* vscale) {
    const int c = blockIdx.x;
    if (c >= TP) return;
    if (unit || c >= T) {
        if (threadIdx.x == 0) vscale[c] = unit_scale;
        return;
    }
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < N; i += blockDim.x) {
        const double x = V[(int64_t)c * ldv + i];
        acc += x * x;
    }
    __shared__ double red[8];
    acc = warp_sum(acc);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        const double nrm = sqrt(s);
        float sc = 1.f;
        if (nrm > 0.0) sc = ldexpf(1.f, (int)floor(log2(sqrt((double)N) / nrm)));
        vscale[c] = sc;
    }
}

// One thread per (column, 8 consecutive rows): scaled V split into the
// B-operand layout.  Columns come in launch groups of tpg; group g holds
// [tile][part][col/8][K-core][col%8][row%8] at vblk + g * (Npad/64) * 2 tpg 128.
// TF32: V rounded to TF32, one part, [tile][col/8][K-core of 4 rows][col%8]
// [row%4] (core matrices of 8 columns x 16 bytes; same tile size).
template <bool HALF, bool TF32 = false>
__device__ __forceinline__ void tc_split_v_body(const float* V, int64_t ldv, int T, int TP, int tpg, int64_t Npad,
                                                const float* vscale, uint8_t* vblk, int64_t idx,
                                                const float* lz_q = nullptr, const float* lz_sco = nullptr) {
    const int64_t groups = Npad / 8;
    if (idx >= groups * TP) return;
    const int c = (int)(idx / groups);
    const int64_t j0 = (idx % groups) * 8;
    float x[8];
    if (c < T) {
        float4 a = *reinterpret_cast<const float4*>(V + (int64_t)c * ldv + j0);
        float4 b = *reinterpret_cast<const float4*>(V + (int64_t)c * ldv + j0 + 4);
        if (lz_sco && lz_sco[(int64_t)c * kScoStride] == 0.f) {
            // The previous step's q_{j+1} = (p - alpha q_j) / beta_{j+1}, in the
            // recurrence step's operation order, stored over p.
            const float* sc = lz_sco + (int64_t)c * kScoStride;
            const float ah = sc[1], al = sc[2], ib = sc[3];
            const float4 qa = *reinterpret_cast<const float4*>(lz_q + (int64_t)c * ldv + j0);
            const float4 qb = *reinterpret_cast<const float4*>(lz_q + (int64_t)c * ldv + j0 + 4);
            float pv[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
            const float qv[8] = {qa.x, qa.y, qa.z, qa.w, qb.x, qb.y, qb.z, qb.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) pv[e] = fmaf(-al, qv[e], fmaf(-ah, qv[e], pv[e])) * ib;
            a = make_float4(pv[0], pv[1], pv[2], pv[3]);
            b = make_float4(pv[4], pv[5], pv[6], pv[7]);
            float4* dst = reinterpret_cast<float4*>(const_cast<float*>(V) + (int64_t)c * ldv + j0);
            dst[0] = a;
            dst[1] = b;
        }
        const float s = vscale[c];
        x[0] = a.x * s; x[1] = a.y * s; x[2] = a.z * s; x[3] = a.w * s;
        x[4] = b.x * s; x[5] = b.y * s; x[6] = b.z * s; x[7] = b.w * s;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0.f;
    }
    const int g = c / tpg, cl = c % tpg;
    const int64_t tile_bytes = 2 * (int64_t)tpg * 128;
    uint8_t* base = vblk + (int64_t)g * (Npad / kTcBN) * tile_bytes + (j0 / kTcBN) * tile_bytes;
    const int jj = (int)(j0 % kTcBN);
    if constexpr (TF32) {
        const int64_t o = (int64_t)(cl >> 3) * 2048 + (jj >> 2) * 128 + (cl & 7) * 16;
        *reinterpret_cast<uint4*>(base + o) = make_uint4(to_tf32(x[0]), to_tf32(x[1]), to_tf32(x[2]), to_tf32(x[3]));
        *reinterpret_cast<uint4*>(base + o + 128) =
            make_uint4(to_tf32(x[4]), to_tf32(x[5]), to_tf32(x[6]), to_tf32(x[7]));
    } else {
        uint32_t h[4], l[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) split_pair<HALF>(x[2 * e], x[2 * e + 1], h[e], l[e]);
        const int64_t off = (int64_t)(cl >> 3) * 1024 + (jj >> 3) * 128 + (cl & 7) * 16;
        *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
        *reinterpret_cast<uint4*>(base + (int64_t)tpg * 128 + off) = make_uint4(l[0], l[1], l[2], l[3]);
    }
}

template <bool HALF, bool TF32>
__global__ void tc_split_v_kernel(const float* V, int64_t ldv, int T, int TP, int tpg, int64_t Npad,
                                  const float* vscale, uint8_t* vblk, const float* lz_q, const float* lz_sco) {
    tc_split_v_body<HALF, TF32>(V, ldv, T, TP, tpg, Npad, vscale, vblk,
                                (int64_t)blockIdx.x * blockDim.x + threadIdx.x, lz_q, lz_sco);
}

// The kernel walks K's columns in steps of kTcKN = 128 (two 64-row operand
// tiles).  Every tcgen05.commit costs about 200 cycles of a serial commit
// path, so a step carries exactly two: one when its S is complete, one when
// its product is complete; each completion barrier has several waiters.
constexpr int kTcKN = 128;
constexpr int kXStep = 2 * kXBytes;              // points of one step, 12 KiB
constexpr int kTcXStages = 3;
template <int TP>
__host__ __device__ constexpr int tc_vstages() {
    return TP <= 32 ? 4 : 3;
}
template <int TP>
__host__ __device__ constexpr int tc_vstep_bytes() {
    return 2 * (2 * TP * 128);                   // two 64-row tiles of split V
}
constexpr int kRing = 8;                         // completion barriers per kind (>= stages + 2)

// Steps of K's columns accumulated in TMEM before the partial sum is folded
// into the compensated running sum (bounds the tensor core's FP32
// accumulation to kTcChunk x 16 MMAs per partial sum).  Fewer steps per fold
// cost exp-warpgroup time (the fold reads TP columns of O) but lower the MVM
// error, and the solves need fewer iterations.  Measured on the 50,000-point
// RBF problem:
//   TP = 64, K^{1/2} with error bound 1e-3: 16 steps, 4.8e-6 MVM error, 915
//     iterations; 12 steps, 3.7e-6 and 897, fastest; 8 steps, 897 but
//     slower; 32 steps, 9.7e-6 and 1000;
//   TP = 32 (a fold reads half as many columns), the 512-problem batch with
//     residual 1e-4: 12 steps, 108 columns left at the iteration cap; 8
//     steps, 77 and 4 % faster; 6, 67 and 4 % faster again; 4 steps, 34 at
//     the same speed as 6.  The 8-column K^{-1/2} solve: 2833, 2704, 2650 and
//     2581 iterations, 2249, 2223, 2235 and 2306 ms.  With the running sum in
//     registers: 3 steps, 23 columns at the cap and 0.6 % faster than 4; 2
//     steps, 17 and 0.8 % slower than 4.  Batched and single solves share the
//     interval (their results are equal bit for bit).
template <int TP>
__host__ __device__ constexpr int tc_chunk() {
    return TP <= 32 ? 3 : 12;
}

// TMEM: three S buffers of 128 columns, each overwritten by its P in place,
// block by block: the 16 values of S in columns [16k, 16k+16) become 8
// columns of leading parts [16k, 16k+8) and 8 of trailing parts [16k+8,
// 16k+16) (two 16-bit values per column), the A operand of K-step k of the
// product; the O accumulator [384, 384 + 2 TP): the three split products of
// a K-step are two MMAs, P_hi [V_hi; V_lo] (N = 2 TP: the leading and
// trailing parts of V are adjacent in the operand layout) and P_lo V_hi
// (N = TP) accumulated into the first half, so O = D[0, TP) + D[TP, 2 TP)
// (measured: 8 N=128 + 8 N=64 MMAs take 29 % less pipe time than 24 N=64).
// Step t uses buffer t % 3, so S(t+2) can be
// computed while the products of steps t-1 and t are still queued; exp
// warpgroup g turns columns [64 g, 64 g + 64) of every step into P.  The
// compensated running sum (leading and trailing FP32 parts) lives in the
// fold threads' registers, one row and TP / 2 columns per thread (measured:
// 3.4 % less time per MVM than a running sum in shared memory).
constexpr int kNB = 3;
constexpr uint32_t kTmemCols = 512;

template <int TP>
__host__ __device__ constexpr int tc_smem_bytes() {
    return kUBytes + kTcXStages * kXStep + tc_vstages<TP>() * tc_vstep_bytes<TP>() + 512;
}

// Barrier slots in shared memory.
enum TcBar {
    kBarU = 0,             // U tile landed
    kBarXFull = 1,         // [4] points of a step landed
    kBarVFull = 5,         // [6] V of a step landed
    kBarSDone = 11,        // [8] S of step t complete (ring t % 8): exp may start, point stage free
    kBarODone = 19,        // [8] product of step t complete: S buffer and V stage free, O readable
    kBarPFull = 27,        // [3] P written over S in buffer b by both exp warpgroups
    kBarOFree = 30,        // O accumulator read out for folding, free again
    kBarDrain = 31,        // [2] every MMA of an issuing thread complete (teardown)
    kBarCount = 33
};

// Kernel value / outputscale from S = -c^2 r^2 / 2 (RBF: S <= 0 up to
// rounding, and ex2 of a rounding-level positive S is harmless).
template <int KT>
__device__ __forceinline__ float p_of_s(float S) {
    if (KT == CIQ_RBF) return ex2_approx(S);
    const float a = sqrt_approx(fmaxf(-10.f * S, 0.f));
    return fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f) * ex2_approx(a * (float)(-kLog2e));
}

// 16 values of S (one TMEM block of a row) -> P split into 8 packed leading
// and 8 packed trailing 16-bit pairs (TF32: the 16 values of P rounded to
// TF32, the first 8 in hi and the last 8 in lo, so the block keeps its
// column order).
template <int KT, bool HALF, bool TF32 = false>
__device__ __forceinline__ void exp_block(const uint32_t (&s)[16], uint32_t (&hi)[8], uint32_t (&lo)[8]) {
    if constexpr (TF32) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            hi[e] = to_tf32(p_of_s<KT>(__uint_as_float(s[e])));
            lo[e] = to_tf32(p_of_s<KT>(__uint_as_float(s[8 + e])));
        }
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const float pa = p_of_s<KT>(__uint_as_float(s[2 * e]));
            const float pb = p_of_s<KT>(__uint_as_float(s[2 * e + 1]));
            split_pair<HALF>(pa, pb, hi[e], lo[e]);
        }
    }
}

// --------------------------------------------------------------- kernel --
// Warp roles (384 threads): warp 0 lane 0 issues the bulk copies, warp 1
// lane 0 the products, warp 2 lane 0 the S MMAs; warps 4-7 and 8-11 are two
// exp warpgroups that split every step's 128 columns between them, fold
// each completed chunk of O into the running sum and write the CTA's column
// sums.  Columns [c0, c0 + TP) of V (those below a.T) are handled.
//
// Split K: with p.nsplit = S, CTA b takes row tile b / S and the steps
// [(b % S) nt / S, (b % S + 1) nt / S) of K's columns, so the grid fills the
// SMs' waves evenly.  Every CTA writes its partial O as (leading, trailing)
// float pairs; tc_finish_body adds a tile's S partials in split order and
// runs the epilogue, in a kernel of its own (one block per row tile) so
// this kernel holds only the pipeline.
template <int KT, int TP, bool HALF, bool TF32 = false>
__device__ __forceinline__ void mvm_tc_body(const TcPoints& p, const MvmArgs<float>& a, int c0, int64_t tile,
                                            int split) {
    // Stopped columns, or an earlier MVM of this call gave up a bounded wait
    // (its results are invalid; the call reports CIQ_ERR_TIMEOUT): no work.
    // One thread reads the flags so the whole CTA takes the same branch.
    __shared__ int skip_all;
    if (threadIdx.x == 0) skip_all = (a.stop && *a.stop) || *p.err;
    __syncthreads();
    if (skip_all) return;
    constexpr int NX = kTcXStages;
    constexpr int NV = tc_vstages<TP>();
    constexpr int VSTEP = tc_vstep_bytes<TP>();
    constexpr int VHALF = VSTEP / 2;                     // one 64-row tile of split V
    static_assert(NX + 2 <= kRing && NV + 2 <= kRing, "completion rings too short");
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sU = smem;
    uint8_t* sX0 = sU + kUBytes;
    uint8_t* sV0 = sX0 + NX * kXStep;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sV0 + NV * VSTEP);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kBarCount);
    volatile int* serr = reinterpret_cast<volatile int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = p.nsplit;
    const int ntot = (int)(a.Npad / kTcKN);
    const int st0 = (int)((int64_t)split * ntot / S);
    const int nt = (int)((int64_t)(split + 1) * ntot / S) - st0;   // steps of this CTA (>= 1)
    constexpr int kTcChunk = tc_chunk<TP>();
    constexpr uint32_t IDESC_S = tc::idesc_f16(kTcBM, kTcKN, !HALF);
    constexpr uint32_t IDESC_O = tc::idesc_f16(kTcBM, TP, !HALF);
    constexpr uint32_t IDESC_O2 = tc::idesc_f16(kTcBM, 2 * TP, !HALF);
    constexpr uint32_t IDESC_T = tc::idesc_tf32(kTcBM, TP);

    if (tid == 0) {
        tc::mbar_init(&bars[kBarU], 1);
        for (int s = 0; s < NX; ++s) tc::mbar_init(&bars[kBarXFull + s], 1);
        for (int s = 0; s < NV; ++s) tc::mbar_init(&bars[kBarVFull + s], 1);
        for (int r = 0; r < kRing; ++r) {
            tc::mbar_init(&bars[kBarSDone + r], 1);
            tc::mbar_init(&bars[kBarODone + r], 1);
        }
        for (int b = 0; b < kNB; ++b) tc::mbar_init(&bars[kBarPFull + b], 256);
        tc::mbar_init(&bars[kBarOFree], 256);
        tc::mbar_init(&bars[kBarDrain], 1);
        tc::mbar_init(&bars[kBarDrain + 1], 1);
        tc::fence_mbarrier_init();
        *serr = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tO0 = tmem + kNB * kTcKN;              // O accumulator, 2 TP columns
    const uint8_t* vblk = p.vblk;
    // Exp warps: compensated running sum (leading, trailing FP32 parts) of
    // the TP / 2 columns this thread folds, for its row, in registers.
    float acc_h[TP / 2], acc_l[TP / 2];
#pragma unroll
    for (int i = 0; i < TP / 2; ++i) acc_h[i] = acc_l[i] = 0.f;

    if (warp == 0) {
        // ---------------------------------------------------------- loader
        // Fixed order: the points of step t + 2 (S runs two
        // steps ahead of the product), then the V of step t.  The point
        // stage of step u was read by S(u - NX), the V stage by the product
        // of step t - NV; each wait is bounded.
        // The whole warp runs the loop; one elected lane issues the copies.
        auto uni = [&](bool b) { return __shfl_sync(0xffffffffu, (int)b, 0) != 0; };
        if (tc::elect_one()) {
            tc::mbar_expect_tx(&bars[kBarU], kUBytes);
            tc::bulk_g2s(sU, p.ua + tile * kUBytes, kUBytes, &bars[kBarU]);
        }
        auto load_x = [&](int u) -> bool {
            const int sx = u % NX;
            if (p.inject && u == 0 && blockIdx.x == 0) return false;   // testing: the copy never comes
            if (u >= NX && !uni(tc::mbar_wait(&bars[kBarSDone + (u - NX) % kRing],
                                              (uint32_t)(((u - NX) / kRing) & 1), kWaitLimit)))
                return false;
            if (tc::elect_one()) {
                tc::mbar_expect_tx(&bars[kBarXFull + sx], kXStep);
                tc::bulk_g2s(sX0 + sx * kXStep, p.ub + (int64_t)(st0 + u) * kXStep, kXStep, &bars[kBarXFull + sx]);
            }
            __syncwarp();
            return true;
        };
        int nx = 0, nv = 0;                               // copies issued
        bool ok = load_x(0);
        nx += ok;
        if (ok && nt > 1) nx += (ok = load_x(1));
        for (int t = 0; ok && t < nt; ++t) {
            if (t + 2 < nt) {
                if (!load_x(t + 2)) { ok = false; break; }
                ++nx;
            }
            const int sv = t % NV;
            if (t >= NV && !uni(tc::mbar_wait(&bars[kBarODone + (t - NV) % kRing],
                                              (uint32_t)(((t - NV) / kRing) & 1), kWaitLimit))) {
                ok = false;
                break;
            }
            if (tc::elect_one()) {
                tc::mbar_expect_tx(&bars[kBarVFull + sv], VSTEP);
                tc::bulk_g2s(sV0 + sv * VSTEP, vblk + (int64_t)(st0 + t) * VSTEP, VSTEP, &bars[kBarVFull + sv]);
            }
            __syncwarp();
            ++nv;
            if (uni(*serr)) break;
        }
        if (!ok && lane == 0) *serr = 1;
        // No copy may land in shared memory after the CTA has left: wait
        // (bounded) for the last copy issued to every stage.
        tc::mbar_wait(&bars[kBarU], 0, kWaitLimit);
        for (int u = max(nx - NX, 0); u < nx; ++u)
            tc::mbar_wait(&bars[kBarXFull + u % NX], (uint32_t)((u / NX) & 1), kWaitLimit);
        for (int u = max(nv - NV, 0); u < nv; ++u)
            tc::mbar_wait(&bars[kBarVFull + u % NV], (uint32_t)((u / NV) & 1), kWaitLimit);
        __syncwarp();
    } else if (warp == 1 || warp == 2) {
        // ----------------------------------------------------- MMA issuers
        // Two warps feed the tensor pipe, so neither's barrier waits leave it
        // idle: warp 2 issues S(h) into buffer h % 3 as soon as the product
        // of step h - 3 (the buffer's last reader) is complete and the
        // points are in; warp 1 issues O += P(t) V(t) once both exp
        // warpgroups have written P(t), V(t) is in and, at the start of a
        // chunk, the accumulator has been folded.  The whole warp runs the
        // loop (so the descriptors are warp-uniform values) and one elected
        // lane issues.  Before leaving, the warp waits (bounded) for all of
        // its MMAs, so tensor memory is never freed under a running MMA.
        auto uni = [&](bool b) { return __shfl_sync(0xffffffffu, (int)b, 0) != 0; };
        bool good = true;
        if (warp == 2) {
            const uint64_t dU = tc::smem_desc(tc::smem_u32(sU), 128, 768);
            const uint64_t dX = tc::smem_desc(tc::smem_u32(sX0), 128, 768);
            // With at most 8 features only K-core 0 of each chunk is
            // non-zero: a K-core stride of one chunk (256 bytes) makes one
            // K16 MMA read core 0 of chunks 0 and 1, U_h [X_h; X_l].
            const uint64_t dU2 = tc::smem_desc(tc::smem_u32(sU), 256, 768);
            const uint64_t dX2 = tc::smem_desc(tc::smem_u32(sX0), 256, 768);
            const bool narrow = p.narrow != 0;
            good = uni(tc::mbar_wait(&bars[kBarU], 0, kWaitLimit));
            for (int h = 0; good && h < nt; ++h) {
                const int sx = h % NX;
                good = uni((h < kNB || tc::mbar_wait(&bars[kBarODone + (h - kNB) % kRing],
                                                     (uint32_t)(((h - kNB) / kRing) & 1), kWaitLimit)) &&
                           tc::mbar_wait(&bars[kBarXFull + sx], (uint32_t)((h / NX) & 1), kWaitLimit));
                if (!good) break;
                tc::fence_after_sync();
                const uint64_t dx = dX + (uint64_t)((sx * kXStep) >> 4);
                const uint32_t tS = tmem + (h % kNB) * kTcKN;
                if (tc::elect_one()) {
                    if (narrow) {
                        tc::mma_f16(tS, dU2, dX2 + (uint64_t)((sx * kXStep) >> 4), IDESC_S, 0u);
                        tc::mma_f16(tS, dU + (uint64_t)(512 >> 4), dx + (uint64_t)(512 >> 4), IDESC_S, 1u);
                    } else {
#pragma unroll
                        for (int ch = 0; ch < 3; ++ch)
                            tc::mma_f16(tS, dU + (uint64_t)((ch * 256) >> 4), dx + (uint64_t)((ch * 256) >> 4),
                                        IDESC_S, ch > 0 ? 1u : 0u);
                    }
                    tc::mma_commit(&bars[kBarSDone + h % kRing]);
                }
                __syncwarp();
                good = uni(!*serr);
            }
        } else {
            // TF32: V's core matrices are 8 columns x 4 rows; 16 K-cores per
            // group of 8 columns of a 64-row tile.
            const uint64_t dV = tc::smem_desc(tc::smem_u32(sV0), 128, TF32 ? 2048 : 1024);
            for (int t = 0; good && t < nt; ++t) {
                const int b = t % kNB, sv = t % NV;
                const int ch = t / kTcChunk;
                const bool fresh = (t % kTcChunk) == 0;
                good = uni(tc::mbar_wait(&bars[kBarPFull + b], (uint32_t)((t / kNB) & 1), kWaitLimit) &&
                           tc::mbar_wait(&bars[kBarVFull + sv], (uint32_t)((t / NV) & 1), kWaitLimit) &&
                           (!fresh || ch < 1 ||
                            tc::mbar_wait(&bars[kBarOFree], (uint32_t)((ch - 1) & 1), kWaitLimit)));
                if (!good) break;
                tc::fence_after_sync();
                const uint32_t tP = tmem + b * kTcKN;
                const uint64_t dv = dV + (uint64_t)((sv * VSTEP) >> 4);
                if (tc::elect_one()) {
                    if (TF32) {
#pragma unroll
                        for (int kk = 0; kk < 16; ++kk) {   // K = 8 columns of P per MMA
                            const uint64_t vb = dv + (uint64_t)(((kk >> 3) * VHALF + (kk & 7) * 256) >> 4);
                            tc::mma_tf32_ts(tO0, tP + kk * 8, vb, IDESC_T, (!fresh || kk > 0) ? 1u : 0u);
                        }
                    } else {
#pragma unroll
                        for (int kk = 0; kk < 8; ++kk) {
                            const uint64_t vb = dv + (uint64_t)(((kk >> 2) * VHALF + (kk & 3) * 256) >> 4);
                            tc::mma_f16_ts(tO0, tP + kk * 16, vb, IDESC_O2, (!fresh || kk > 0) ? 1u : 0u);   // P_hi [V_hi; V_lo]
                            tc::mma_f16_ts(tO0, tP + kk * 16 + 8, vb, IDESC_O, 1u);                          // P_lo V_hi
                        }
                    }
                    tc::mma_commit(&bars[kBarODone + t % kRing]);
                }
                __syncwarp();
                good = uni(!*serr);
            }
        }
        if (!good && lane == 0) *serr = 1;
        if (tc::elect_one()) tc::mma_commit(&bars[kBarDrain + (warp - 1)]);
        __syncwarp();
        tc::mbar_wait(&bars[kBarDrain + (warp - 1)], 0, kWaitLimit);
        __syncwarp();
    } else if (warp >= 4) {
        // --------------------------------------------------- exp warpgroups
        const int g = (warp - 4) >> 2;                    // columns [64 g, 64 g + 64) of every step
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int r = 32 * (warp & 3) + lane;             // row of the tile = TMEM lane
        for (int t = 0; t < nt; ++t) {
            const int b = t % kNB;
            const uint32_t tS = tmem + b * kTcKN + g * 64 + lane_base;
            const bool good = tc::mbar_wait(&bars[kBarSDone + t % kRing], (uint32_t)((t / kRing) & 1), kWaitLimit);
            if (__shfl_sync(0xffffffffu, (int)(!good || *serr), 0)) { *serr = 1; break; }
            tc::fence_after_sync();
            // S in four 16-column blocks; the load of block k+1 is in flight
            // while block k is turned into P, written back over the columns
            // block k was read from.
            uint32_t A[16], B[16];
            uint32_t h0[8], l0[8], h1[8], l1[8], h2[8], l2[8], h3[8], l3[8];
            tc::tmem_ld16(tS, A);
            tc::tmem_wait_ld16(A);
            tc::tmem_ld16(tS + 16, B);
            exp_block<KT, HALF, TF32>(A, h0, l0);
            tc::tmem_st8(tS, h0);
            tc::tmem_st8(tS + 8, l0);
            tc::tmem_wait_ld16(B);
            tc::tmem_ld16(tS + 32, A);
            exp_block<KT, HALF, TF32>(B, h1, l1);
            tc::tmem_st8(tS + 16, h1);
            tc::tmem_st8(tS + 24, l1);
            tc::tmem_wait_ld16(A);
            tc::tmem_ld16(tS + 48, B);
            exp_block<KT, HALF, TF32>(A, h2, l2);
            tc::tmem_st8(tS + 32, h2);
            tc::tmem_st8(tS + 40, l2);
            tc::tmem_wait_ld16(B);
            exp_block<KT, HALF, TF32>(B, h3, l3);
            tc::tmem_st8(tS + 48, h3);
            tc::tmem_st8(tS + 56, l3);
            tc::tmem_wait_st64(h0, l0, h1, l1, h2, l2, h3, l3);
            tc::fence_before_sync();
            tc::mbar_arrive(&bars[kBarPFull + b]);
            // At the start of a chunk, fold the previous chunk of O into the
            // running sum after this step's P is written, so the product of
            // this step waits only for the accumulator to be read, not for
            // the exp work as well; each warpgroup takes half of the
            // columns, and the accumulator is released as soon as it has
            // been read.
            if (t >= kTcChunk && (t % kTcChunk) == 0) {
                const int te = t - 1;                     // last step of the chunk
                const bool okc = tc::mbar_wait(&bars[kBarODone + te % kRing], (uint32_t)((te / kRing) & 1), kWaitLimit);
                if (__shfl_sync(0xffffffffu, (int)(!okc || *serr), 0)) { *serr = 1; break; }
                tc::fence_after_sync();
                constexpr int HB = TP / 2 / 16;           // 16-column blocks per warpgroup
#pragma unroll
                for (int cb = 0; cb < HB; ++cb) {
                    const int col0 = g * (TP / 2) + 16 * cb;
                    uint32_t oa[16], ob[16];
                    tc::tmem_ld16(tO0 + lane_base + col0, oa);
                    if (!TF32) tc::tmem_ld16(tO0 + TP + lane_base + col0, ob);
                    tc::tmem_wait_ld16(oa);
                    if (!TF32) tc::tmem_wait_ld16(ob);
                    if (cb == HB - 1) {
                        tc::fence_before_sync();
                        tc::mbar_arrive(&bars[kBarOFree]);
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        two_sum_into(acc_h[16 * cb + e], acc_l[16 * cb + e], __uint_as_float(oa[e]));
                        if (!TF32) two_sum_into(acc_h[16 * cb + e], acc_l[16 * cb + e], __uint_as_float(ob[e]));
                    }
                }
            }
        }
    }

    // ------------------------------------------------------- partial sums
    // Warpgroup g writes the columns it folded, [g TP / 2, (g + 1) TP / 2):
    // running sum + the last chunk's two accumulator halves, formed as a
    // float pair and rounded once to a float (2^-24 relative, far below the
    // error of the 16-bit split operands; halves the finishing traffic).
    if (warp >= 4) {
        const int g = (warp - 4) >> 2;
        const int r = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const bool good = !*serr && tc::mbar_wait(&bars[kBarODone + (nt - 1) % kRing],
                                                  (uint32_t)(((nt - 1) / kRing) & 1), kWaitLimit);
        const bool ok = !__shfl_sync(0xffffffffu, (int)(!good || *serr), 0);
        if (!ok) *serr = 1;
        tc::fence_after_sync();
        float* part = p.part + ((int64_t)tile * S + split) * TP * kTcBM;
#pragma unroll
        for (int cb = 0; cb < TP / 32; ++cb) {
            const int col0 = g * (TP / 2) + 16 * cb;
            uint32_t oa[16], ob[16];
            if (ok) {
                tc::tmem_ld16(tO0 + lane_base + col0, oa);
                if (!TF32) tc::tmem_ld16(tO0 + TP + lane_base + col0, ob);
                tc::tmem_wait_ld16(oa);
                if (!TF32) tc::tmem_wait_ld16(ob);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int cl = col0 + e;
                float h = 0.f, l = 0.f;
                if (ok) {
                    h = acc_h[16 * cb + e];
                    l = acc_l[16 * cb + e];
                }
                if (ok) {
                    two_sum_into(h, l, __uint_as_float(oa[e]));
                    if (!TF32) two_sum_into(h, l, __uint_as_float(ob[e]));
                }
                part[cl * kTcBM + r] = h + l;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *serr) atomicExch(p.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

template <int KT, int TP, bool HALF, bool TF32>
__global__ void __launch_bounds__(384, 1) mvm_tc_kernel(TcPoints p, MvmArgs<float> a, int c0) {
    mvm_tc_body<KT, TP, HALF, TF32>(p, a, c0, blockIdx.x / p.nsplit, blockIdx.x % p.nsplit);
}

// ------------------------------------------------------------- finish --
// Rows [128 tile, 128 tile + 128) and columns [16 cg, 16 cg + 16) of O: the
// S split partials of every entry added in split order (2Sum into a
// (leading, trailing) float pair), scaled by outscale / vscale, plus
// sigma^2 V, then the epilogue of `a`: kPlain stores O; kLanczos writes
// p = O - beta q_prev over q_prev and forms the tile's q.p, p.p, q.q per
// column.  128 threads: thread t takes column t / 8 and the 16 consecutive
// rows 16 (t % 8) ..., loads them as float4s, sums its products (exact by
// FMA) as float pairs and meets the other 7 threads of its column in three
// shuffles; the pair is converted to FP64 once (FP64 runs at a few
// operations per clock per SM on this part).
constexpr int kFinCols = 16;
template <int TP>
__device__ __forceinline__ void tc_finish_body(const TcPoints& p, const MvmArgs<float>& a, int c0, int64_t tile,
                                               int cg) {
    const int tid = threadIdx.x;
    const int cbeg = cg * kFinCols, cend = min(cbeg + kFinCols, a.T - c0);
    if (cbeg >= cend) return;                             // columns past T: nothing to do
    // Threads of columns past T keep their lanes in the shuffles but touch
    // no memory (whole 8-thread groups, never a partial one).
    const bool active = cbeg + (tid >> 3) < cend;
    const int cl = active ? cbeg + (tid >> 3) : cbeg;    // column of the group
    const int r0 = 16 * (tid & 7);                        // first of this thread's rows
    const int c = c0 + cl;
    const float sc = a.s / p.vscale[c];                   // exact: vscale is a power of two
    const bool lanczos = a.mode == kLanczos;
    const float bt = lanczos ? (float)a.beta[c] : 0.f;
    const int S = p.nsplit;
    const float* part = p.part + (int64_t)tile * S * TP * kTcBM + (int64_t)cl * kTcBM + r0;
    const int64_t i0 = tile * kTcBM + r0;
    const int64_t base = (int64_t)c * a.ldv + i0;
    float* pdst = a.pout ? a.pout : a.qprev;              // p: over q_{j-1} unless pout is set
    float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int half = 0; half < 2 && active; ++half) {
        // 8 rows: every load issued before any use.
        float h[8], l[8], v[8], qp[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) { h[e] = 0.f; l[e] = 0.f; }
        for (int sp = 0; sp < S; ++sp) {
            const float4* src = reinterpret_cast<const float4*>(part + (int64_t)sp * TP * kTcBM + 8 * half);
            const float4 x0 = __ldcg(src), x1 = __ldcg(src + 1);
            const float xs[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
            for (int e = 0; e < 8; ++e) two_sum_into(h[e], l[e], xs[e]);
        }
        {
            const float4* vs = reinterpret_cast<const float4*>(a.V + base + 8 * half);
            const float4 v0 = vs[0], v1 = vs[1];
            v[0] = v0.x; v[1] = v0.y; v[2] = v0.z; v[3] = v0.w; v[4] = v1.x; v[5] = v1.y; v[6] = v1.z; v[7] = v1.w;
        }
        if (lanczos) {
            const float4* qs = reinterpret_cast<const float4*>(a.qprev + base + 8 * half);
            const float4 q0 = qs[0], q1 = qs[1];
            qp[0] = q0.x; qp[1] = q0.y; qp[2] = q0.z; qp[3] = q0.w; qp[4] = q1.x; qp[5] = q1.y; qp[6] = q1.z; qp[7] = q1.w;
        }
        float o[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            o[e] = fmaf(h[e], sc, l[e] * sc);
            o[e] += a.noise * v[e];
        }
        if (!lanczos) {
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                const int64_t i = i0 + 8 * half + e;
                if (i < a.N) a.out[(int64_t)c * a.ldo + i] = o[e];
            }
            continue;
        }
        float pv[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const bool row_in = i0 + 8 * half + e < a.N;
            pv[e] = row_in ? o[e] - bt * qp[e] : 0.f;
            const float fa[3] = {v[e], pv[e], v[e]}, fb[3] = {pv[e], pv[e], v[e]};
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float pr = fa[k] * fb[k];
                two_sum_into(sh[k], sl[k], pr);
                sl[k] += fmaf(fa[k], fb[k], -pr);
            }
        }
        float4* pd = reinterpret_cast<float4*>(pdst + base + 8 * half);
        pd[0] = make_float4(pv[0], pv[1], pv[2], pv[3]);
        pd[1] = make_float4(pv[4], pv[5], pv[6], pv[7]);
    }
    if (!lanczos) return;
    // The 8 threads of a column are consecutive lanes of one warp.
#pragma unroll
    for (int ofs = 1; ofs < 8; ofs <<= 1) {
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float oh = __shfl_xor_sync(0xffffffffu, sh[k], ofs);
            const float ol = __shfl_xor_sync(0xffffffffu, sl[k], ofs);
            two_sum_into(sh[k], sl[k], oh);
            sl[k] += ol;
        }
    }
    if (active && (tid & 7) == 0) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            a.partials[((int64_t)tile * a.T + c) * 3 + k] = (double)sh[k] + (double)sl[k];
    }
}

template <int TP>
__global__ void __launch_bounds__(128) tc_finish_kernel(TcPoints p, MvmArgs<float> a, int c0) {
    if ((a.stop && *a.stop) || *p.err) return;      // the product launch before it is complete
    tc_finish_body<TP>(p, a, c0, blockIdx.x / (TP / kFinCols), blockIdx.x % (TP / kFinCols));
}

// ------------------------------------------------------ batched problems --
// Block b takes item b of a work list of (problem, row tile x split); the
// problem's operands and MVM arguments are copied to shared memory and the
// same body runs as for one problem.  One launch covers both kernel types:
// the CTA's problem selects the body (a branch uniform over the CTA), so RBF
// and Matern problems share one work list and fill the same waves.
template <int TP, bool HALF>
__global__ void __launch_bounds__(384, 1) batched_tc_mvm_kernel(const BatchProblem* probs, DevList L, int parity,
                                                                 int pre) {
    int pb, local;
    if (!list_item(L, blockIdx.x, pb, local)) return;
    __shared__ TcPoints sp;
    __shared__ MvmArgs<float> sa;
    if (threadIdx.x == 0) {
        sp = probs[pb].tcp;
        sa = pre ? probs[pb].pre[parity] : probs[pb].mvm[parity];
    }
    __syncthreads();
    if (sa.kt == CIQ_RBF) mvm_tc_body<CIQ_RBF, TP, HALF>(sp, sa, 0, local / sp.nsplit, local % sp.nsplit);
    else mvm_tc_body<CIQ_MATERN52, TP, HALF>(sp, sa, 0, local / sp.nsplit, local % sp.nsplit);
}

// Block b finishes item `local` (row tile x 16-column group) of problem pb.
template <int TP>
__global__ void __launch_bounds__(128) batched_tc_finish_kernel(const BatchProblem* probs, DevList L, int parity,
                                                                int pre) {
    int pb, local;
    if (!list_item(L, blockIdx.x, pb, local)) return;
    __shared__ TcPoints sp;
    __shared__ MvmArgs<float> sa;
    if (threadIdx.x == 0) {
        sp = probs[pb].tcp;
        sa = pre ? probs[pb].pre[parity] : probs[pb].mvm[parity];
    }
    __syncthreads();
    if ((sa.stop && *sa.stop) || *sp.err) return;
    tc_finish_body<TP>(sp, sa, 0, local / (TP / kFinCols), local % (TP / kFinCols));
}

// One block per problem: centre of the points, unit V scales, cleared
// error flag.
__global__ void __launch_bounds__(256) batched_tc_mean_kernel(const BatchProblem* probs, DevList L) {
    int pb, local;
    if (!list_item(L, blockIdx.x, pb, local)) return;
    const BatchProblem& bp = probs[pb];
    const TcPoints& tp = bp.tcp;
    const MvmArgs<float>& m = bp.mvm[0];
    tc_mean_body(m.X, m.N, m.dp, tp.mean);
    const float unit_scale = ldexpf(1.f, (int)floor(0.5 * log2((double)m.N)));
    for (int c = threadIdx.x; c < tp.TP; c += 256) tp.vscale[c] = unit_scale;
    if (threadIdx.x == 0) *tp.err = 0;
}

template <bool HALF>
__global__ void __launch_bounds__(256) batched_tc_points_kernel(const BatchProblem* probs, DevList L) {
    int pb, local;
    if (!list_item(L, blockIdx.x, pb, local)) return;
    const BatchProblem& bp = probs[pb];
    const MvmArgs<float>& m = bp.mvm[0];
    const double c2 = m.kt == CIQ_RBF ? kLog2e : 1.0;
    tc_points_body<HALF>(m.X, m.N, m.Npad, m.dp, bp.d, (float)sqrt(c2), (float)(0.5 * c2), bp.tcp.mean, bp.tcp.ua,
                         bp.tcp.ub, (int64_t)local * 256 + threadIdx.x);
}

// The pre-pass (one column) uses a 32-column group, as a single solve does.
template <bool HALF>
__global__ void __launch_bounds__(256) batched_tc_split_kernel(const BatchProblem* probs, DevList L, int parity,
                                                               int pre) {
    int pb, local;
    if (!list_item(L, blockIdx.x, pb, local)) return;
    const BatchProblem& bp = probs[pb];
    const MvmArgs<float>& m = pre ? bp.pre[parity] : bp.mvm[parity];
    if (m.stop && *m.stop) return;
    const TcPoints& tp = bp.tcp;
    const int tpw = pre ? 32 : tp.TP;
    tc_split_v_body<HALF>(m.V, m.ldv, m.T, tpw, tpw, tp.Npad, tp.vscale, tp.vblk, (int64_t)local * 256 + threadIdx.x);
}

// ------------------------------------------------ stored K on tensor cores --
// O = K V for a K held in device memory (FP32, row-major, leading dimension
// ldk, padded rows and columns zero) on the product pipeline of the
// on-the-fly MVM, with K's tile in place of P.  Every step's 128 x 64 tile
// arrives by TMA as two 32-column boxes with the 128-byte swizzle (the
// split warps read rows, which then fall in different banks); the split
// warpgroups scale it by a power of two (so max_i K_ii, which bounds every
// |K_ij| of a positive semidefinite K, sits at 2^14), split it into 16-bit
// leading and trailing parts in a TMEM buffer and release the stage; the
// product warp multiplies the buffer with the split V.  K is read from
// device memory once per MVM.
constexpr int kStKN = 64;                          // columns of K per step
constexpr int kStKStages = 3;
constexpr int kStKBytes = kTcBM * kStKN * 4;       // 32 KiB: two 16 KiB boxes
constexpr int kStNB = 4;                           // P buffers of 64 TMEM columns
constexpr int kStVStages = 3;
template <int TP>
__host__ __device__ constexpr int st_vstep_bytes() {
    return 2 * TP * 128;                           // one 64-row tile of split V
}
// Steps per fold: 1,536 columns (TP = 64), as in the on-the-fly kernel, or 512 (TP <= 32).
template <int TP>
__host__ __device__ constexpr int st_chunk() {
    return TP <= 32 ? 8 : 24;
}
template <int TP>
__host__ __device__ constexpr int st_smem_bytes() {
    return 1024 + kStKStages * kStKBytes + kStVStages * st_vstep_bytes<TP>() + 512;
}
enum StBar {
    kSbKFull = 0,      // [3] tile of K landed
    kSbKEmpty = 3,     // [3] the split warps have read the stage
    kSbVFull = 6,      // [3] V of a step landed
    kSbPFull = 9,      // [4] split K written to buffer b
    kSbODone = 17,     // [8] product of step t complete
    kSbOFree = 25,     // O accumulator read out for folding
    kSbDrain = 26,     // every MMA complete (teardown)
    kSbCount = 27
};

template <int TP, bool HALF>
__global__ void __launch_bounds__(384, 1) stored_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcPoints p,
                                                           MvmArgs<float> a, int c0, float kscale) {
    __shared__ int skip_all;
    if (threadIdx.x == 0) skip_all = (a.stop && *a.stop) || *p.err;
    __syncthreads();
    if (skip_all) return;
    constexpr int VSTEP = st_vstep_bytes<TP>();
    constexpr int C = st_chunk<TP>();
    extern __shared__ __align__(1024) uint8_t st_smem[];
    // The swizzled boxes need 1024-byte aligned stages (1024 bytes reserved).
    uint8_t* sK = st_smem + ((1024u - (tc::smem_u32(st_smem) & 1023u)) & 1023u);
    uint8_t* sV = sK + kStKStages * kStKBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sV + kStVStages * VSTEP);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kSbCount);
    volatile int* serr = reinterpret_cast<volatile int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int S = p.nsplit;
    const int64_t tile = blockIdx.x / S;
    const int split = blockIdx.x % S;
    const int64_t i0 = tile * kTcBM;
    const int ntot = (int)(a.Npad / kStKN);
    const int st0 = (int)((int64_t)split * ntot / S);
    const int nt = (int)((int64_t)(split + 1) * ntot / S) - st0;   // steps of this CTA (>= 1)
    constexpr uint32_t IDESC_O = tc::idesc_f16(kTcBM, TP, !HALF);
    constexpr uint32_t IDESC_O2 = tc::idesc_f16(kTcBM, 2 * TP, !HALF);

    if (tid == 0) {
        for (int s = 0; s < kStKStages; ++s) {
            tc::mbar_init(&bars[kSbKFull + s], 1);
            tc::mbar_init(&bars[kSbKEmpty + s], 256);
        }
        for (int s = 0; s < kStVStages; ++s) tc::mbar_init(&bars[kSbVFull + s], 1);
        for (int b = 0; b < kStNB; ++b) tc::mbar_init(&bars[kSbPFull + b], 256);
        for (int r = 0; r < kRing; ++r) tc::mbar_init(&bars[kSbODone + r], 1);
        tc::mbar_init(&bars[kSbOFree], 256);
        tc::mbar_init(&bars[kSbDrain], 1);
        tc::fence_mbarrier_init();
        *serr = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, kTmemCols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tO0 = tmem + kStNB * kStKN;            // O accumulator, 2 TP columns
    // Exp warps: compensated running sum (leading, trailing FP32 parts) of
    // the TP / 2 columns this thread folds, for its row, in registers.
    float acc_h[TP / 2], acc_l[TP / 2];
#pragma unroll
    for (int i = 0; i < TP / 2; ++i) acc_h[i] = acc_l[i] = 0.f;
    auto uni = [&](bool b) { return __shfl_sync(0xffffffffu, (int)b, 0) != 0; };

    if (warp == 0) {
        // ---------------------------------------------------------- loader
        // The tile of step t goes to stage t % 3 once the split warps have
        // read step t - 3; the V of step t once the product of t - 3 is done.
        int nk = 0, nv = 0;
        bool ok = true;
        for (int t = 0; t < nt; ++t) {
            const int sk = t % kStKStages, sv = t % kStVStages;
            if (t >= kStKStages &&
                !uni(tc::mbar_wait(&bars[kSbKEmpty + sk], (uint32_t)(((t - kStKStages) / kStKStages) & 1), kWaitLimit))) {
                ok = false;
                break;
            }
            const int x = (st0 + t) * kStKN;              // a multiple of 64 columns: 16-byte aligned
            if (tc::elect_one()) {
                tc::mbar_expect_tx(&bars[kSbKFull + sk], kStKBytes);
                tc::tma_load_2d(sK + sk * kStKBytes, &tmap, x, (int)i0, &bars[kSbKFull + sk]);
                tc::tma_load_2d(sK + sk * kStKBytes + kStKBytes / 2, &tmap, x + 32, (int)i0, &bars[kSbKFull + sk]);
            }
            __syncwarp();
            ++nk;
            if (t >= kStVStages &&
                !uni(tc::mbar_wait(&bars[kSbODone + (t - kStVStages) % kRing],
                                   (uint32_t)(((t - kStVStages) / kRing) & 1), kWaitLimit))) {
                ok = false;
                break;
            }
            if (tc::elect_one()) {
                tc::mbar_expect_tx(&bars[kSbVFull + sv], VSTEP);
                tc::bulk_g2s(sV + sv * VSTEP, p.vblk + (int64_t)(st0 + t) * VSTEP, VSTEP, &bars[kSbVFull + sv]);
            }
            __syncwarp();
            ++nv;
            if (uni(*serr)) break;
        }
        if (!ok && lane == 0) *serr = 1;
        // No copy may land in shared memory after the CTA has left.
        for (int u = max(nk - kStKStages, 0); u < nk; ++u)
            tc::mbar_wait(&bars[kSbKFull + u % kStKStages], (uint32_t)((u / kStKStages) & 1), kWaitLimit);
        for (int u = max(nv - kStVStages, 0); u < nv; ++u)
            tc::mbar_wait(&bars[kSbVFull + u % kStVStages], (uint32_t)((u / kStVStages) & 1), kWaitLimit);
        __syncwarp();
    } else if (warp == 1) {
        // --------------------------------------------------- product issuer
        bool good = true;
        const uint64_t dV = tc::smem_desc(tc::smem_u32(sV), 128, 1024);
        for (int t = 0; good && t < nt; ++t) {
            const int b = t % kStNB, sv = t % kStVStages;
            const int ch = t / C;
            const bool fresh = (t % C) == 0;
            good = uni(tc::mbar_wait(&bars[kSbPFull + b], (uint32_t)((t / kStNB) & 1), kWaitLimit) &&
                       tc::mbar_wait(&bars[kSbVFull + sv], (uint32_t)((t / kStVStages) & 1), kWaitLimit) &&
                       (!fresh || ch < 1 || tc::mbar_wait(&bars[kSbOFree], (uint32_t)((ch - 1) & 1), kWaitLimit)));
            if (!good) break;
            tc::fence_after_sync();
            const uint32_t tP = tmem + b * kStKN;
            const uint64_t dv = dV + (uint64_t)((sv * VSTEP) >> 4);
            if (tc::elect_one()) {
#pragma unroll
                for (int kk = 0; kk < 4; ++kk) {
                    const uint64_t vb = dv + (uint64_t)((kk * 256) >> 4);
                    tc::mma_f16_ts(tO0, tP + kk * 16, vb, IDESC_O2, (!fresh || kk > 0) ? 1u : 0u);   // K_hi [V_hi; V_lo]
                    tc::mma_f16_ts(tO0, tP + kk * 16 + 8, vb, IDESC_O, 1u);                          // K_lo V_hi
                }
                tc::mma_commit(&bars[kSbODone + t % kRing]);
            }
            __syncwarp();
            good = uni(!*serr);
        }
        if (!good && lane == 0) *serr = 1;
        if (tc::elect_one()) tc::mma_commit(&bars[kSbDrain]);
        __syncwarp();
        tc::mbar_wait(&bars[kSbDrain], 0, kWaitLimit);
        __syncwarp();
    } else if (warp >= 4) {
        // ------------------------------------------------ split warpgroups
        // Warpgroup g takes columns [32 g, 32 g + 32) of every step (box g);
        // thread r takes row r of the tile (TMEM lane r).
        const int g = (warp - 4) >> 2;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const int r = 32 * (warp & 3) + lane;
        for (int t = 0; t < nt; ++t) {
            const int sk = t % kStKStages, b = t % kStNB;
            bool good = tc::mbar_wait(&bars[kSbKFull + sk], (uint32_t)((t / kStKStages) & 1), kWaitLimit);
            // Buffer b was last read by the product of step t - 4.
            if (good && t >= kStNB)
                good = tc::mbar_wait(&bars[kSbODone + (t - kStNB) % kRing], (uint32_t)(((t - kStNB) / kRing) & 1),
                                     kWaitLimit);
            if (__shfl_sync(0xffffffffu, (int)(!good || *serr), 0)) { *serr = 1; break; }
            tc::fence_after_sync();
            // Row r of box g: 16-byte chunk j of the row sits at chunk j ^ (r % 8).
            const uint8_t* row = sK + sk * kStKBytes + g * (kStKBytes / 2) + r * 128;
            float x[32];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const float4 v = *reinterpret_cast<const float4*>(row + ((j ^ (r & 7)) << 4));
                x[4 * j] = v.x * kscale;
                x[4 * j + 1] = v.y * kscale;
                x[4 * j + 2] = v.z * kscale;
                x[4 * j + 3] = v.w * kscale;
            }
            tc::mbar_arrive(&bars[kSbKEmpty + sk]);
            uint32_t h0[8], l0[8], h1[8], l1[8];
#pragma unroll
            for (int e = 0; e < 8; ++e) {
                split_pair<HALF>(x[2 * e], x[2 * e + 1], h0[e], l0[e]);
                split_pair<HALF>(x[16 + 2 * e], x[17 + 2 * e], h1[e], l1[e]);
            }
            const uint32_t tS = tmem + b * kStKN + g * 32 + lane_base;
            tc::tmem_st8(tS, h0);
            tc::tmem_st8(tS + 8, l0);
            tc::tmem_st8(tS + 16, h1);
            tc::tmem_st8(tS + 24, l1);
            tc::tmem_wait_st32(h0, l0, h1, l1);
            tc::fence_before_sync();
            tc::mbar_arrive(&bars[kSbPFull + b]);
            // At the start of a chunk, fold the previous chunk of O into the
            // running sum (half of the columns per warpgroup).
            if (t >= C && (t % C) == 0) {
                const int te = t - 1;
                const bool okc = tc::mbar_wait(&bars[kSbODone + te % kRing], (uint32_t)((te / kRing) & 1), kWaitLimit);
                if (__shfl_sync(0xffffffffu, (int)(!okc || *serr), 0)) { *serr = 1; break; }
                tc::fence_after_sync();
                constexpr int HB = TP / 2 / 16;
#pragma unroll
                for (int cb = 0; cb < HB; ++cb) {
                    const int col0 = g * (TP / 2) + 16 * cb;
                    uint32_t oa[16], ob[16];
                    tc::tmem_ld16(tO0 + lane_base + col0, oa);
                    tc::tmem_ld16(tO0 + TP + lane_base + col0, ob);
                    tc::tmem_wait_ld16(oa);
                    tc::tmem_wait_ld16(ob);
                    if (cb == HB - 1) {
                        tc::fence_before_sync();
                        tc::mbar_arrive(&bars[kSbOFree]);
                    }
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        two_sum_into(acc_h[16 * cb + e], acc_l[16 * cb + e], __uint_as_float(oa[e]));
                        two_sum_into(acc_h[16 * cb + e], acc_l[16 * cb + e], __uint_as_float(ob[e]));
                    }
                }
            }
        }
    }

    // ------------------------------------------------------- partial sums
    if (warp >= 4) {
        const int g = (warp - 4) >> 2;
        const int r = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const bool good = !*serr && tc::mbar_wait(&bars[kSbODone + (nt - 1) % kRing],
                                                  (uint32_t)(((nt - 1) / kRing) & 1), kWaitLimit);
        const bool ok = !__shfl_sync(0xffffffffu, (int)(!good || *serr), 0);
        if (!ok) *serr = 1;
        tc::fence_after_sync();
        float* part = p.part + ((int64_t)tile * S + split) * TP * kTcBM;
#pragma unroll
        for (int cb = 0; cb < TP / 32; ++cb) {
            const int col0 = g * (TP / 2) + 16 * cb;
            uint32_t oa[16], ob[16];
            if (ok) {
                tc::tmem_ld16(tO0 + lane_base + col0, oa);
                tc::tmem_ld16(tO0 + TP + lane_base + col0, ob);
                tc::tmem_wait_ld16(oa);
                tc::tmem_wait_ld16(ob);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const int cl = col0 + e;
                float h = 0.f, l = 0.f;
                if (ok) {
                    h = acc_h[16 * cb + e];
                    l = acc_l[16 * cb + e];
                }
                if (ok) {
                    two_sum_into(h, l, __uint_as_float(oa[e]));
                    two_sum_into(h, l, __uint_as_float(ob[e]));
                }
                part[cl * kTcBM + r] = h + l;
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid == 0 && *serr) atomicExch(p.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, kTmemCols);
}

// Largest diagonal entry of K (bounds every |K_ij| of a PSD matrix), one block.
__global__ void stored_diag_max_kernel(const float* Kmat, int64_t ldk, int64_t N, float* out) {
    __shared__ float red[8];
    float m = 0.f;
    for (int64_t i = threadIdx.x; i < N; i += 256) m = fmaxf(m, fabsf(Kmat[i * ldk + i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 8; ++w) m = fmaxf(m, red[w]);
        out[0] = fmaxf(m, red[0]);
    }
}

// A kernel's shared-memory attribute is set once per device (the attribute
// belongs to the device that is current when it is set); `done` holds one
// bit per device id.
template <typename F>
cudaError_t set_smem_once(std::atomic<uint64_t>& done, F kernel, int smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const uint64_t bit = dev < 64 ? uint64_t(1) << dev : 0;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

template <int KT, int TP, bool HALF, bool TF32>
cudaError_t launch_tp(const TcPoints& p, const MvmArgs<float>& a, int c0, cudaStream_t st) {
    constexpr int smem = tc_smem_bytes<TP>();
    static std::atomic<uint64_t> configured{0};
    cudaError_t e0 = set_smem_once(configured, mvm_tc_kernel<KT, TP, HALF, TF32>, smem);
    if (e0 != cudaSuccess) return e0;
    mvm_tc_kernel<KT, TP, HALF, TF32><<<(unsigned)(a.Npad / kTcBM * p.nsplit), 384, smem, st>>>(p, a, c0);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc_finish_kernel<TP><<<(unsigned)(a.Npad / kTcBM * (TP / kFinCols)), 128, 0, st>>>(p, a, c0);
    return cudaGetLastError();
}

template <int KT, bool HALF>
cudaError_t launch_kt_half(const TcPoints& p, const MvmArgs<float>& a, int tpg, int c0, cudaStream_t st) {
    if (p.tf32) {
        if (!HALF) return cudaErrorInvalidValue;   // TF32 pairs with the FP16 point split
        switch (tpg) {
            case 32: return launch_tp<KT, 32, true, true>(p, a, c0, st);
            case 64: return launch_tp<KT, 64, true, true>(p, a, c0, st);
            default: return cudaErrorInvalidValue;
        }
    }
    switch (tpg) {
        case 32: return launch_tp<KT, 32, HALF, false>(p, a, c0, st);
        case 64: return launch_tp<KT, 64, HALF, false>(p, a, c0, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool tc_supported(int precision, int d) {
    return (precision == CIQ_PREC_BF16 || precision == CIQ_PREC_FP16 || precision == CIQ_PREC_TF32) && d >= 1 &&
           d <= 14;
}

// Columns of V per MVM launch group (T > 64 runs as groups of 64, which
// with the two 128-column S buffers fill TMEM; the TMEM loads and stores
// move 32 columns, so a group is at least 32 wide).
int tc_group_t(int T) {
    if (T <= 32) return 32;
    return 64;
}

int tc_padded_t(int T) {
    if (T < 1 || T > 1024) return -1;
    const int g = tc_group_t(T);
    return (T + g - 1) / g * g;
}

int64_t tc_row_tiles(int64_t Npad) { return Npad / kTcBM; }

// CTAs per row tile: the S in 1..8 that minimises waves x steps per CTA,
// with 4 steps charged per CTA for its pipeline start and epilogue.
int tc_split(int64_t Npad) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            sms <= 0) {
            cudaGetLastError();
            sms = 148;
        }
    }
    const int64_t tiles = Npad / kTcBM, steps = Npad / kTcKN;
    int best = 1;
    double best_cost = 1e300;
    for (int S = 1; S <= 8 && S <= steps; ++S) {
        const double waves = (double)((tiles * S + sms - 1) / sms);
        const double cost = waves * ((double)steps / S + 4.0);
        if (cost < best_cost * 0.999) { best_cost = cost; best = S; }
    }
    return best;
}

// max_split 8 means "choose"; a smaller value is used as given (never
// more than the steps of K's columns).
int tc_nsplit(int64_t Npad, int max_split) {
    const int steps = (int)(Npad / kTcKN);
    const int S = max_split >= 8 ? tc_split(Npad) : max_split;
    return std::max(1, std::min(S, steps));
}

size_t tc_points_bytes(int64_t Npad, int T, int max_split) {
    const int TP = tc_padded_t(T);
    if (TP < 0) return 0;
    const size_t pts = (size_t)Npad * kTcRowBytes;
    const size_t vb = (size_t)(Npad / kTcBN) * 2 * TP * 128;
    const int S = tc_nsplit(Npad, max_split);
    const size_t part = (size_t)(Npad / kTcBM) * S * tc_group_t(T) * kTcBM * sizeof(float) + 256;
    return 2 * pts + vb + 256 * 4 + (size_t)TP * sizeof(float) + 16 * sizeof(double) + 256 + part;
}

TcPoints tc_points_layout(char* base, int64_t Npad, int T, int precision, int max_split, int d) {
    TcPoints p;
    p.narrow = d + 2 <= 8 ? 1 : 0;
    p.Npad = Npad;
    p.TP = tc_padded_t(T);
    p.half = (precision == CIQ_PREC_FP16 || precision == CIQ_PREC_TF32) ? 1 : 0;
    p.tf32 = precision == CIQ_PREC_TF32 ? 1 : 0;
    auto take = [&](size_t bytes) {
        char* q = base;
        base += (bytes + 255) / 256 * 256;
        return q;
    };
    const size_t pts = (size_t)Npad * kTcRowBytes;
    p.ua = reinterpret_cast<uint8_t*>(take(pts));
    p.ub = reinterpret_cast<uint8_t*>(take(pts));
    p.vblk = reinterpret_cast<uint8_t*>(take((size_t)(Npad / kTcBN) * 2 * p.TP * 128));
    p.vscale = reinterpret_cast<float*>(take((size_t)p.TP * sizeof(float)));
    p.mean = reinterpret_cast<double*>(take(16 * sizeof(double)));
    p.err = reinterpret_cast<int*>(take(sizeof(int)));
    p.nsplit = tc_nsplit(Npad, max_split);
    p.part = reinterpret_cast<float*>(take((size_t)(Npad / kTcBM) * p.nsplit * tc_group_t(T) * kTcBM * sizeof(float)));
    return p;
}

cudaError_t launch_tc_prepare(const TcPoints& p, const float* Xp, int64_t N, int dp, int d, int kt,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.mean, 0, 16 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.err, 0, sizeof(int), st)) != cudaSuccess) return e;
    tc_mean_kernel<<<1, 256, 0, st>>>(Xp, N, dp, p.mean);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    const double c2 = kt == CIQ_RBF ? kLog2e : 1.0;
    const unsigned blocks = (unsigned)((p.Npad + 127) / 128);
    if (p.half)
        tc_points_kernel<true><<<blocks, 128, 0, st>>>(Xp, N, p.Npad, dp, d, (float)sqrt(c2), (float)(0.5 * c2),
                                                       p.mean, p.ua, p.ub);
    else
        tc_points_kernel<false><<<blocks, 128, 0, st>>>(Xp, N, p.Npad, dp, d, (float)sqrt(c2), (float)(0.5 * c2),
                                                        p.mean, p.ua, p.ub);
    return cudaGetLastError();
}

cudaError_t launch_mvm_tc(const TcPoints& p, const MvmArgs<float>& a, bool unit_columns, cudaStream_t st,
                          bool scale_ready) {
    if (p.TP < 0 || a.T > p.TP || a.Npad != p.Npad || a.ldv != a.Npad) return cudaErrorInvalidValue;
    cudaError_t e = cudaSuccess;
    if (!(unit_columns && scale_ready)) {
        const float unit_scale = ldexpf(1.f, (int)floor(0.5 * log2((double)a.N)));
        tc_vscale_kernel<<<p.TP, 256, 0, st>>>(a.V, a.ldv, a.N, a.T, p.TP, unit_scale, unit_columns ? 1 : 0,
                                               p.vscale);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t work = (a.Npad / 8) * p.TP;
    const unsigned vblocks = (unsigned)((work + 255) / 256);
    if (p.tf32)
        tc_split_v_kernel<true, true><<<vblocks, 256, 0, st>>>(a.V, a.ldv, a.T, p.TP, tc_group_t(a.T), a.Npad,
                                                               p.vscale, p.vblk, a.lz_q, a.lz_sco);
    else if (p.half)
        tc_split_v_kernel<true, false><<<vblocks, 256, 0, st>>>(a.V, a.ldv, a.T, p.TP, tc_group_t(a.T), a.Npad,
                                                                p.vscale, p.vblk, a.lz_q, a.lz_sco);
    else
        tc_split_v_kernel<false, false><<<vblocks, 256, 0, st>>>(a.V, a.ldv, a.T, p.TP, tc_group_t(a.T), a.Npad,
                                                                 p.vscale, p.vblk, a.lz_q, a.lz_sco);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // V is split into groups of tpg columns; group g's tiles start at
    // vblk + g * (Npad / 64) * 2 * tpg * 128.
    const int tpg = tc_group_t(a.T);
    for (int c0 = 0; c0 < a.T && e == cudaSuccess; c0 += tpg) {
        TcPoints pg = p;
        pg.vblk = p.vblk + (size_t)(c0 / tpg) * (size_t)(a.Npad / kTcBN) * 2 * tpg * 128;
        if (a.kt == CIQ_RBF)
            e = p.half ? launch_kt_half<CIQ_RBF, true>(pg, a, tpg, c0, st) : launch_kt_half<CIQ_RBF, false>(pg, a, tpg, c0, st);
        else
            e = p.half ? launch_kt_half<CIQ_MATERN52, true>(pg, a, tpg, c0, st)
                       : launch_kt_half<CIQ_MATERN52, false>(pg, a, tpg, c0, st);
    }
    return e;
}

namespace {
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

template <int TP, bool HALF>
cudaError_t launch_st_tp(const CUtensorMap& tmap, const TcPoints& p, const MvmArgs<float>& a, int c0, float kscale,
                         cudaStream_t st) {
    constexpr int smem = st_smem_bytes<TP>();
    static std::atomic<uint64_t> configured{0};
    cudaError_t e0 = set_smem_once(configured, stored_tc_kernel<TP, HALF>, smem);
    if (e0 != cudaSuccess) return e0;
    stored_tc_kernel<TP, HALF><<<(unsigned)(a.Npad / kTcBM * p.nsplit), 384, smem, st>>>(tmap, p, a, c0, kscale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    tc_finish_kernel<TP><<<(unsigned)(a.Npad / kTcBM * (TP / kFinCols)), 128, 0, st>>>(p, a, c0);
    return cudaGetLastError();
}
}  // namespace

float stored_tc_scale(double max_diag) {
    if (!(max_diag > 0.0) || !std::isfinite(max_diag)) return 1.f;
    return ldexpf(1.f, 14 - (int)ceil(log2(max_diag)));
}

cudaError_t launch_stored_diag_max(const float* Kmat, int64_t ldk, int64_t N, float* out, cudaStream_t st) {
    stored_diag_max_kernel<<<1, 256, 0, st>>>(Kmat, ldk, N, out);
    return cudaGetLastError();
}

cudaError_t launch_stored_mvm_tc(const float* Kmat, int64_t ldk, const TcPoints& p, const MvmArgs<float>& args,
                                 float kscale, bool unit_columns, cudaStream_t st, bool scale_ready) {
    if (p.TP < 0 || p.tf32 || args.T > p.TP || args.Npad != p.Npad || args.ldv != args.Npad || ldk % 4 != 0 ||
        ldk < args.Npad || args.Npad % kTcBM != 0 || (reinterpret_cast<uintptr_t>(Kmat) & 15) != 0 || !(kscale > 0.f))
        return cudaErrorInvalidValue;
    MvmArgs<float> a = args;
    a.noise = 0.f;              // the stored matrix holds sigma^2 on its diagonal
    a.s = 1.f / kscale;         // exact: kscale is a power of two
    cudaError_t e = cudaSuccess;
    if (!(unit_columns && scale_ready)) {
        const float unit_scale = ldexpf(1.f, (int)floor(0.5 * log2((double)a.N)));
        tc_vscale_kernel<<<p.TP, 256, 0, st>>>(a.V, a.ldv, a.N, a.T, p.TP, unit_scale, unit_columns ? 1 : 0,
                                               p.vscale);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    const int64_t work = (a.Npad / 8) * p.TP;
    const unsigned vblocks = (unsigned)((work + 255) / 256);
    if (p.half)
        tc_split_v_kernel<true, false><<<vblocks, 256, 0, st>>>(a.V, a.ldv, a.T, p.TP, tc_group_t(a.T), a.Npad,
                                                                p.vscale, p.vblk, a.lz_q, a.lz_sco);
    else
        tc_split_v_kernel<false, false><<<vblocks, 256, 0, st>>>(a.V, a.ldv, a.T, p.TP, tc_group_t(a.T), a.Npad,
                                                                 p.vscale, p.vblk, a.lz_q, a.lz_sco);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // K as a 2-D tensor of Npad x Npad floats, row pitch ldk floats; boxes of
    // 32 columns x 128 rows with the 128-byte swizzle.
    // cuTensorMapEncodeTiled is reached through the runtime's entry-point
    // lookup (the library does not link libcuda).
    static EncodeTiledFn encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q{};
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return cudaErrorNotSupported;
        }
        encode = reinterpret_cast<EncodeTiledFn>(fn);
    }
    CUtensorMap tmap;
    const cuuint64_t dims[2] = {(cuuint64_t)a.Npad, (cuuint64_t)a.Npad};
    const cuuint64_t pitch[1] = {(cuuint64_t)ldk * sizeof(float)};
    const cuuint32_t box[2] = {32, (cuuint32_t)kTcBM};
    const cuuint32_t estride[2] = {1, 1};
    if (encode(&tmap, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(Kmat), dims, pitch, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorInvalidValue;
    const int tpg = tc_group_t(a.T);
    for (int c0 = 0; c0 < a.T && e == cudaSuccess; c0 += tpg) {
        TcPoints pg = p;
        pg.vblk = p.vblk + (size_t)(c0 / tpg) * (size_t)(a.Npad / kTcBN) * 2 * tpg * 128;
        if (tpg == 32) e = p.half ? launch_st_tp<32, true>(tmap, pg, a, c0, kscale, st)
                                  : launch_st_tp<32, false>(tmap, pg, a, c0, kscale, st);
        else e = p.half ? launch_st_tp<64, true>(tmap, pg, a, c0, kscale, st)
                        : launch_st_tp<64, false>(tmap, pg, a, c0, kscale, st);
    }
    return e;
}

cudaError_t launch_batched_tc_mean(const BatchProblem* probs, DevList one, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_tc_mean_kernel<<<blocks, 256, 0, st>>>(probs, one);
    return cudaGetLastError();
}

cudaError_t launch_batched_tc_points(const BatchProblem* probs, DevList rows256, int blocks, bool half,
                                     cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (half) batched_tc_points_kernel<true><<<blocks, 256, 0, st>>>(probs, rows256);
    else batched_tc_points_kernel<false><<<blocks, 256, 0, st>>>(probs, rows256);
    return cudaGetLastError();
}

cudaError_t launch_batched_tc_split(const BatchProblem* probs, int parity, DevList L, int blocks, bool half,
                                    bool pre, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (half) batched_tc_split_kernel<true><<<blocks, 256, 0, st>>>(probs, L, parity, pre ? 1 : 0);
    else batched_tc_split_kernel<false><<<blocks, 256, 0, st>>>(probs, L, parity, pre ? 1 : 0);
    return cudaGetLastError();
}

namespace {
template <int TP, bool HALF>
cudaError_t configure_btc() {
    static std::atomic<uint64_t> configured{0};
    return set_smem_once(configured, batched_tc_mvm_kernel<TP, HALF>, tc_smem_bytes<TP>());
}

template <int TP, bool HALF>
cudaError_t launch_btc(const BatchProblem* probs, int parity, int pre, DevList L, int blocks, cudaStream_t st) {
    cudaError_t e = configure_btc<TP, HALF>();
    if (e != cudaSuccess) return e;
    batched_tc_mvm_kernel<TP, HALF><<<blocks, 384, tc_smem_bytes<TP>(), st>>>(probs, L, parity, pre);
    return cudaGetLastError();
}

template <bool HALF>
cudaError_t configure_btc_all(int TP) {
    return TP == 32 ? configure_btc<32, HALF>() : configure_btc<64, HALF>();
}
template <bool HALF>
cudaError_t launch_btc_tp(const BatchProblem* probs, int TP, int parity, int pre, DevList L, int blocks,
                         cudaStream_t st) {
    return TP == 32 ? launch_btc<32, HALF>(probs, parity, pre, L, blocks, st)
                    : launch_btc<64, HALF>(probs, parity, pre, L, blocks, st);
}
}  // namespace

cudaError_t prepare_batched_tc_mvm(int TP, bool half) {
    if (TP != 32 && TP != 64) return cudaErrorInvalidValue;
    return half ? configure_btc_all<true>(TP) : configure_btc_all<false>(TP);
}

cudaError_t launch_batched_tc_mvm(const BatchProblem* probs, int TP, bool half, int parity, bool pre, DevList L,
                                  int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    if (TP != 32 && TP != 64) return cudaErrorInvalidValue;
    const int pr = pre ? 1 : 0;
    return half ? launch_btc_tp<true>(probs, TP, parity, pr, L, blocks, st)
                : launch_btc_tp<false>(probs, TP, parity, pr, L, blocks, st);
}

cudaError_t launch_batched_tc_finish(const BatchProblem* probs, int TP, int parity, bool pre, DevList L, int blocks,
                                     cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    const int pr = pre ? 1 : 0;
    if (TP == 32) batched_tc_finish_kernel<32><<<blocks, 128, 0, st>>>(probs, L, parity, pr);
    else if (TP == 64) batched_tc_finish_kernel<64><<<blocks, 128, 0, st>>>(probs, L, parity, pr);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

}  // namespace ciq
