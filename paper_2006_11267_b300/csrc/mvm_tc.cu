// On-the-fly kernel MVM on the tcgen05 tensor cores (sm_103a).
//
// O = (K_XX + sigma^2 I) V without storing K (the map-reduce MVM of Sec. 3.3).
// One CTA owns 128 rows of K and streams the points and V in tiles of 64:
//
//   S   = U_i V_j^T on tensor cores, kind::f16, accumulator in TMEM.  Rows are
//         augmented, u = [c(x - m), -c^2 |x - m|^2 / 2, 1] and v = [c(x - m), 1,
//         -c^2 |x - m|^2 / 2], so S = -c^2 r^2 / 2 directly (norm expansion of
//         the distance; m is the centre of the points).  Each operand is split
//         into a 16-bit leading part and a 16-bit trailing part and S =
//         U_h V_h + U_h V_l + U_l V_h (three K-chunks of one MMA sequence):
//         about 22 significant bits with FP16 parts.
//   P   = k(r) / s from S on the SFU (RBF: ex2(S) with c^2 = log2 e; Matern-5/2:
//         a = sqrt(-10 S), (1 + a + a^2/3) ex2(-a log2 e)), split again into
//         leading/trailing 16-bit parts and written back over S in tensor
//         memory (tcgen05.st), so the product reads its A operand from TMEM
//         and shared-memory bandwidth is left to the B operands and copies.
//   O  += P_h Vt_h + P_h Vt_l + P_l Vt_h on tensor cores, accumulator in TMEM,
//         with Vt = V times a power of two per column, split like U.
//
// The operands are pre-arranged in global memory in the shared-memory layout
// of the MMA, so every tile is one bulk copy (cp.async.bulk) completing on
// an mbarrier, double-buffered.  The epilogue reads O from TMEM and applies
// the same Lanczos epilogue as the CUDA-core MVM.  Every wait is bounded: on
// timeout the CTA records an error flag, skips the rest and frees its TMEM.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <math.h>

#include "mvm_tc.cuh"
#include "tc_ptx.cuh"

namespace ciq {

namespace {

constexpr long long kWaitLimit = 4000000000LL;   // clock cycles, ~2 s at 2 GHz
constexpr int kUBytes = kTcBM * kTcRowBytes;      // 12 KiB
constexpr int kXBytes = kTcBN * kTcRowBytes;      // 6 KiB
constexpr int kPPart = kTcBM * kTcBN * 2;         // 16 KiB per 16-bit part

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

// Convert a pair to 16-bit leading parts (packed) and the trailing parts.
template <bool HALF>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t& hi, uint32_t& lo) {
    if (HALF) {
        const __half2 h = __floats2half2_rn(a, b);
        const float2 f = __half22float2(h);
        const __half2 l = __floats2half2_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        const float2 f = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(a - f.x, b - f.y);
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// ---------------------------------------------------------- operand prep --
__global__ void tc_mean_kernel(const float* Xp, int64_t N, int dp, double* mean) {
    double acc[kMaxDimPad];
#pragma unroll
    for (int k = 0; k < kMaxDimPad; ++k) acc[k] = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N; i += (int64_t)gridDim.x * blockDim.x)
        for (int k = 0; k < dp; ++k) acc[k] += (double)Xp[i * dp + k];
    for (int k = 0; k < dp; ++k) {
        const double v = warp_sum(acc[k]);
        if ((threadIdx.x & 31) == 0) atomicAdd(&mean[k], v / (double)N);
    }
}

// One thread per row: u, v augmented and split, written in the operand layout
// [row/8][chunk 0..2][K-core 0..1][row%8][element%8] (16-bit elements).
template <bool HALF>
__global__ void tc_points_kernel(const float* Xp, int64_t N, int64_t Npad, int dp, int d, float c,
                                 float c2half, const double* mean, uint8_t* ua, uint8_t* ub) {
    const int64_t row = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
    const size_t base = (size_t)(row >> 3) * kTcRowBytes * 8 + (size_t)(row & 7) * 16;
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
#pragma unroll
        for (int kc = 0; kc < 2; ++kc) {
            const uint16_t* a = achunk[ch] + kc * 8;
            const uint16_t* b = bchunk[ch] + kc * 8;
            const size_t off = base + (size_t)ch * 256 + (size_t)kc * 128;
            *reinterpret_cast<uint4*>(ua + off) =
                make_uint4(pack2(a[0], a[1]), pack2(a[2], a[3]), pack2(a[4], a[5]), pack2(a[6], a[7]));
            *reinterpret_cast<uint4*>(ub + off) =
                make_uint4(pack2(b[0], b[1]), pack2(b[2], b[3]), pack2(b[4], b[5]), pack2(b[6], b[7]));
        }
    }
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
template <bool HALF>
__global__ void tc_split_v_kernel(const float* V, int64_t ldv, int T, int TP, int tpg, int64_t Npad,
                                  const float* vscale, uint8_t* vblk) {
    const int64_t groups = Npad / 8;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= groups * TP) return;
    const int c = (int)(idx / groups);
    const int64_t j0 = (idx % groups) * 8;
    float x[8];
    if (c < T) {
        const float4 a = *reinterpret_cast<const float4*>(V + (int64_t)c * ldv + j0);
        const float4 b = *reinterpret_cast<const float4*>(V + (int64_t)c * ldv + j0 + 4);
        const float s = vscale[c];
        x[0] = a.x * s; x[1] = a.y * s; x[2] = a.z * s; x[3] = a.w * s;
        x[4] = b.x * s; x[5] = b.y * s; x[6] = b.z * s; x[7] = b.w * s;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) x[e] = 0.f;
    }
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) split_pair<HALF>(x[2 * e], x[2 * e + 1], h[e], l[e]);
    const int g = c / tpg, cl = c % tpg;
    const int64_t tile_bytes = 2 * (int64_t)tpg * 128;
    uint8_t* base = vblk + (int64_t)g * (Npad / kTcBN) * tile_bytes + (j0 / kTcBN) * tile_bytes;
    const int jj = (int)(j0 % kTcBN);
    const int64_t off = (int64_t)(cl >> 3) * 1024 + (jj >> 3) * 128 + (cl & 7) * 16;
    *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
    *reinterpret_cast<uint4*>(base + (int64_t)tpg * 128 + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// Separate rings for the point tiles (released when S is computed) and the
// V tiles (released when the product with P completes), as deep as shared
// memory allows, so the bulk copies run well ahead of the MMAs.
constexpr int kTcXStages = 8;
template <int TP>
__host__ __device__ constexpr int tc_vstages() {
    return TP <= 64 ? 8 : 4;
}

// Tiles of K's columns accumulated in TMEM before the partial sum is folded
// into the compensated running sum (keeps the tensor core's FP32 accumulation
// to 16 x 4 x 3 = 192 steps per partial sum).
constexpr int kTcChunk = 16;

// TMEM: NB S buffers of 64 columns, each overwritten by its P (leading part
// in the first 32 columns, trailing part in the next 32, two 16-bit values
// per column); O [64 NB, 64 NB + TP); running sum leading part
// [64 NB + TP, 64 NB + 2 TP) and trailing part [64 NB + 2 TP, 64 NB + 3 TP).
// Four S/P buffers when they fit (T <= 64), two otherwise: tile t uses
// buffer t % NB and exp warpgroup t % 2, so each buffer serves one
// warpgroup and its barrier phases advance one at a time.
template <int TP>
__host__ __device__ constexpr int tc_sbuffers() {
    return (4 * kTcBN + 3 * TP <= 512) ? 4 : 2;
}

template <int TP>
__host__ __device__ constexpr uint32_t tmem_cols() {
    return (tc_sbuffers<TP>() * kTcBN + 3 * TP <= 256) ? 256u : 512u;
}

template <int TP>
__host__ __device__ constexpr int tc_smem_bytes() {
    return kUBytes + kTcXStages * kXBytes + tc_vstages<TP>() * (2 * TP * 128) + 512;
}

// Barrier slots in shared memory.
enum TcBar {
    kBarU = 0,             // U tile landed
    kBarXFull = 1,         // [8] point tile landed
    kBarXFree = 9,         // [8] point tile consumed by S
    kBarVFull = 17,        // [8] V tile landed
    kBarVFree = 25,        // [8] V tile consumed by the product
    kBarSFull = 33,        // [4] S buffer written by the MMA
    kBarSFree = 37,        // [4] S/P buffer released by the product that read P
    kBarPFull = 41,        // [4] P written over S by its exp warpgroup
    kBarOChunk = 45,       // a chunk of O is complete (to be folded)
    kBarOFree = 46,        // O folded into the running sum, accumulator free
    kBarOFull = 47,        // last chunk of O complete
    kBarCount = 48
};

// Kernel value / outputscale from S = -c^2 r^2 / 2 (RBF: S <= 0 up to
// rounding, and ex2 of a rounding-level positive S is harmless).
template <int KT>
__device__ __forceinline__ float p_of_s(float S) {
    if (KT == CIQ_RBF) return ex2_approx(S);
    const float a = sqrt_approx(fmaxf(-10.f * S, 0.f));
    return fmaf(a, fmaf(a, 1.0f / 3.0f, 1.0f), 1.0f) * ex2_approx(a * (float)(-kLog2e));
}

// --------------------------------------------------------------- kernel --
// Warp roles (384 threads): warp 0 lane 0 issues the bulk copies, warp 1
// lane 0 issues the MMAs, warps 4-7 and 8-11 are two exp warpgroups taking
// even and odd tiles (S and P double-buffered).  Warps 8-11 also fold each
// completed chunk of O into the running sum; warps 4-7 run the epilogue.
// Tensor pipe order: S(t) = U X_t^T, then O += P(t-1) V(t-1), so the exp of
// one tile overlaps the products of its neighbours.  Columns [c0, c0 + TP)
// of V (those below a.T) are handled.
template <int KT, int TP, bool HALF>
__global__ void __launch_bounds__(384, 1) mvm_tc_kernel(TcPoints p, MvmArgs<float> a, int c0) {
    if (a.stop && *a.stop) return;
    constexpr int NX = kTcXStages;
    constexpr int NV = tc_vstages<TP>();
    constexpr int NB = tc_sbuffers<TP>();
    constexpr int VBYTES = 2 * TP * 128;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* sU = smem;
    uint8_t* sX0 = sU + kUBytes;
    uint8_t* sV0 = sX0 + NX * kXBytes;
    uint64_t* bars = reinterpret_cast<uint64_t*>(sV0 + NV * VBYTES);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bars + kBarCount);
    volatile int* serr = reinterpret_cast<volatile int*>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t tile = blockIdx.x;
    const int64_t i0 = tile * kTcBM;
    const int nt = (int)(a.Npad / kTcBN);
    const int nfold = (nt - 1) / kTcChunk;               // chunks folded before the last one
    constexpr uint32_t NCOLS = tmem_cols<TP>();
    constexpr uint32_t IDESC_S = tc::idesc_f16(kTcBM, kTcBN, !HALF);
    constexpr uint32_t IDESC_O = tc::idesc_f16(kTcBM, TP, !HALF);

    if (tid == 0) {
        tc::mbar_init(&bars[kBarU], 1);
        for (int s = 0; s < NX; ++s) {
            tc::mbar_init(&bars[kBarXFull + s], 1);
            tc::mbar_init(&bars[kBarXFree + s], 1);
        }
        for (int s = 0; s < NV; ++s) {
            tc::mbar_init(&bars[kBarVFull + s], 1);
            tc::mbar_init(&bars[kBarVFree + s], 1);
        }
        for (int b = 0; b < NB; ++b) {
            tc::mbar_init(&bars[kBarSFull + b], 1);
            tc::mbar_init(&bars[kBarSFree + b], 1);
            tc::mbar_init(&bars[kBarPFull + b], 128);
        }
        tc::mbar_init(&bars[kBarOChunk], 1);
        tc::mbar_init(&bars[kBarOFree], 128);
        tc::mbar_init(&bars[kBarOFull], 1);
        tc::fence_mbarrier_init();
        *serr = 0;
    }
    if (warp == 0) {
        tc::tmem_alloc(tslot, NCOLS);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t tO = tmem + NB * kTcBN;
    const uint32_t tRh = tO + TP;
    const uint32_t tRl = tO + 2 * TP;
    const uint8_t* vblk = p.vblk;

    if (warp == 0) {
        // ---------------------------------------------------------- loader
        // Two independent rings, polled without blocking: point tile tx
        // waits for S(tx - NX) to free its stage, V tile tv for the product
        // of tile tv - NV.  The whole warp runs the loop (uniform control
        // flow, addresses in uniform registers); one elected lane issues.
        {
            const bool leader = tc::elect_one();
            if (leader) {
                tc::mbar_expect_tx(&bars[kBarU], kUBytes);
                tc::bulk_g2s(sU, p.ua + tile * kUBytes, kUBytes, &bars[kBarU]);
            }
            __syncwarp();
            int tx = 0, tv = 0;
            long long last = clock64();
            while (tx < nt || tv < nt) {
                if (__shfl_sync(0xffffffffu, (int)*serr, 0)) break;
                bool progressed = false;
                if (tx < nt) {
                    const int st = tx % NX;
                    const bool ok = tx < NX || tc::mbar_test(&bars[kBarXFree + st], (uint32_t)((tx / NX - 1) & 1));
                    if (__shfl_sync(0xffffffffu, (int)ok, 0)) {
                        if (tc::elect_one()) {
                            tc::mbar_expect_tx(&bars[kBarXFull + st], kXBytes);
                            tc::bulk_g2s(sX0 + st * kXBytes, p.ub + (int64_t)tx * kXBytes, kXBytes,
                                         &bars[kBarXFull + st]);
                        }
                        __syncwarp();
                        ++tx;
                        progressed = true;
                    }
                }
                if (tv < nt) {
                    const int st = tv % NV;
                    const bool ok = tv < NV || tc::mbar_test(&bars[kBarVFree + st], (uint32_t)((tv / NV - 1) & 1));
                    if (__shfl_sync(0xffffffffu, (int)ok, 0)) {
                        if (tc::elect_one()) {
                            tc::mbar_expect_tx(&bars[kBarVFull + st], VBYTES);
                            tc::bulk_g2s(sV0 + st * VBYTES, vblk + (int64_t)tv * VBYTES, VBYTES, &bars[kBarVFull + st]);
                        }
                        __syncwarp();
                        ++tv;
                        progressed = true;
                    }
                }
                if (progressed) last = clock64();
                else if (__shfl_sync(0xffffffffu, (int)(clock64() - last > kWaitLimit), 0)) {
                    if (lane == 0) *serr = 1;
                    break;
                }
            }
        }
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        // Event-driven: S(g1) = U X^T is issued as soon as its S buffer and
        // point tile are ready, O += P(g2) V(g2) as soon as P(g2) and its V
        // tile are ready; S is preferred so the in-order tensor pipe never
        // waits behind a product whose P is late.  Each barrier's next phase
        // can only complete after this warp issues the matching MMA, so parity
        // tests are unambiguous; test_wait never suspends the warp.  The whole
        // warp runs the loop with uniform control flow, so the descriptors
        // stay in uniform registers; one elected lane issues each MMA.
        {
            const uint32_t aU = tc::smem_u32(sU);
            bool good = tc::mbar_wait(&bars[kBarU], 0, kWaitLimit);
            good = __shfl_sync(0xffffffffu, (int)good, 0) != 0;
            int g1 = 0, g2 = 0;
            long long last = clock64();
            while (good && g2 < nt) {
                if (__shfl_sync(0xffffffffu, (int)*serr, 0)) { good = false; break; }
                bool progressed = false;
                if (g1 < nt) {
                    const int st = g1 % NX, b = g1 % NB;
                    const bool ok = tc::mbar_test(&bars[kBarXFull + st], (uint32_t)((g1 / NX) & 1)) &&
                                    (g1 < NB || tc::mbar_test(&bars[kBarSFree + b], (uint32_t)((g1 / NB - 1) & 1)));
                    if (__shfl_sync(0xffffffffu, (int)ok, 0)) {
                        tc::fence_after_sync();
                        const uint32_t aX = tc::smem_u32(sX0 + st * kXBytes);
                        const uint32_t tS = tmem + b * kTcBN;
                        if (tc::elect_one()) {
#pragma unroll
                            for (int ch = 0; ch < 3; ++ch)
                                tc::mma_f16(tS, tc::smem_desc(aU + ch * 256, 128, 768),
                                            tc::smem_desc(aX + ch * 256, 128, 768), IDESC_S, ch > 0 ? 1u : 0u);
                            tc::mma_commit(&bars[kBarSFull + b]);
                            tc::mma_commit(&bars[kBarXFree + st]);
                        }
                        __syncwarp();
                        ++g1;
                        progressed = true;
                    }
                }
                if (!progressed && g2 < g1) {
                    const int bu = g2 % NB, su = g2 % NV;
                    const bool fresh = (g2 % kTcChunk) == 0;
                    const bool ok = tc::mbar_test(&bars[kBarPFull + bu], (uint32_t)((g2 / NB) & 1)) &&
                                    tc::mbar_test(&bars[kBarVFull + su], (uint32_t)((g2 / NV) & 1)) &&
                                    (!fresh || g2 == 0 ||
                                     tc::mbar_test(&bars[kBarOFree], (uint32_t)((g2 / kTcChunk - 1) & 1)));
                    if (__shfl_sync(0xffffffffu, (int)ok, 0)) {
                        tc::fence_after_sync();
                        const uint32_t tP = tmem + bu * kTcBN;     // P over S: hi cols [0,32), lo [32,64)
                        const uint32_t aV = tc::smem_u32(sV0 + su * VBYTES);
                        if (tc::elect_one()) {
#pragma unroll
                            for (int g = 0; g < 3; ++g) {
                                const uint32_t pa = tP + (g == 2 ? 32 : 0);
                                const uint32_t vb = aV + (g == 1 ? TP * 128 : 0);
#pragma unroll
                                for (int kk = 0; kk < 4; ++kk)
                                    tc::mma_f16_ts(tO, pa + kk * 8, tc::smem_desc(vb + kk * 256, 128, 1024), IDESC_O,
                                                   (!fresh || g > 0 || kk > 0) ? 1u : 0u);
                            }
                            tc::mma_commit(&bars[kBarSFree + bu]);
                            tc::mma_commit(&bars[kBarVFree + su]);
                            if ((g2 % kTcChunk) == kTcChunk - 1 && g2 != nt - 1) tc::mma_commit(&bars[kBarOChunk]);
                        }
                        __syncwarp();
                        ++g2;
                        progressed = true;
                    }
                }
                if (progressed) last = clock64();
                else if (__shfl_sync(0xffffffffu, (int)(clock64() - last > kWaitLimit), 0)) good = false;
            }
            if (good && tc::elect_one()) tc::mma_commit(&bars[kBarOFull]);
            __syncwarp();
            if (!good && lane == 0) *serr = 1;
        }
    } else if (warp >= 4) {
        // --------------------------------------------------- exp warpgroups
        const int g = (warp - 4) >> 2;                    // 0: even tiles, 1: odd tiles
        const int r = 32 * (warp & 3) + lane;             // row in the tile = TMEM lane
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int t = g; t < nt; t += 2) {
            const int b = t % NB;
            const uint32_t tS = tmem + b * kTcBN + lane_base;
            const bool good = tc::mbar_wait(&bars[kBarSFull + b], (uint32_t)((t / NB) & 1), kWaitLimit);
            if (__shfl_sync(0xffffffffu, (int)(!good || *serr), 0)) { *serr = 1; break; }
            tc::fence_after_sync();
            uint32_t s0[32], s1[32];
            tc::tmem_ld32(tS, s0);
            tc::tmem_ld32(tS + 32, s1);
            uint32_t hq[32], lq[32];
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float pa = p_of_s<KT>(__uint_as_float(s0[2 * e]));
                const float pb = p_of_s<KT>(__uint_as_float(s0[2 * e + 1]));
                split_pair<HALF>(pa, pb, hq[e], lq[e]);
            }
#pragma unroll
            for (int e = 0; e < 16; ++e) {
                const float pa = p_of_s<KT>(__uint_as_float(s1[2 * e]));
                const float pb = p_of_s<KT>(__uint_as_float(s1[2 * e + 1]));
                split_pair<HALF>(pa, pb, hq[16 + e], lq[16 + e]);
            }
            // P over S in tensor memory: 64 values per row -> 32 columns per part.
            tc::tmem_st32(tS, hq);
            tc::tmem_st32(tS + 32, lq);
            tc::fence_before_sync();
            tc::mbar_arrive(&bars[kBarPFull + b]);
            // Fold a completed chunk of O into the running sum (odd warpgroup).
            if (g == 1 && (t % kTcChunk) == kTcChunk - 1 && t != nt - 1) {
                const int c = t / kTcChunk;
                const bool okc = tc::mbar_wait(&bars[kBarOChunk], (uint32_t)(c & 1), kWaitLimit);
                if (__shfl_sync(0xffffffffu, (int)(!okc || *serr), 0)) { *serr = 1; break; }
                tc::fence_after_sync();
#pragma unroll 1
                for (int cc = 0; cc < TP / 32; ++cc) {
                    uint32_t o[32], rh[32], rl[32];
                    tc::tmem_ld32(tO + lane_base + 32 * cc, o);
                    if (c > 0) {
                        tc::tmem_ld32(tRh + lane_base + 32 * cc, rh);
                        tc::tmem_ld32(tRl + lane_base + 32 * cc, rl);
                    }
#pragma unroll
                    for (int e = 0; e < 32; ++e) {
                        float h = c > 0 ? __uint_as_float(rh[e]) : 0.f;
                        float l = c > 0 ? __uint_as_float(rl[e]) : 0.f;
                        two_sum_into(h, l, __uint_as_float(o[e]));
                        rh[e] = __float_as_uint(h);
                        rl[e] = __float_as_uint(l);
                    }
                    tc::tmem_st32(tRh + lane_base + 32 * cc, rh);
                    tc::tmem_st32(tRl + lane_base + 32 * cc, rl);
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&bars[kBarOFree]);
            }
        }
    }

    // ------------------------------------------------------------ epilogue
    double* red = reinterpret_cast<double*>(sX0);         // [4 warps][TP][3], free once O is complete
    if (warp >= 4 && warp < 8) {
        const int r = 32 * (warp & 3) + lane;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        const bool good = !*serr && tc::mbar_wait(&bars[kBarOFull], 0, kWaitLimit);
        const bool ok = !__shfl_sync(0xffffffffu, (int)(!good || *serr), 0);
        if (!ok) *serr = 1;
        tc::fence_after_sync();
        const int64_t i = i0 + r;
        const double outscale = a.s;
        const int wl = warp & 3;
#pragma unroll 1
        for (int cc = 0; cc < TP / 32; ++cc) {
            uint32_t o[32], rh[32], rl[32];
            if (ok) {
                tc::tmem_ld32(tO + lane_base + 32 * cc, o);
                if (nfold > 0) {
                    tc::tmem_ld32(tRh + lane_base + 32 * cc, rh);
                    tc::tmem_ld32(tRl + lane_base + 32 * cc, rl);
                }
            }
#pragma unroll 1
            for (int e = 0; e < 32; ++e) {
                const int cl = 32 * cc + e;
                const int c = c0 + cl;
                if (c >= a.T) break;
                double qp = 0.0, pp = 0.0, qq = 0.0;
                if (ok) {
                    double sum = (double)__uint_as_float(o[e]);
                    if (nfold > 0) sum += (double)__uint_as_float(rh[e]) + (double)__uint_as_float(rl[e]);
                    const float val = (float)(sum * (outscale / (double)p.vscale[c]));
                    lanczos_epilogue_value(a, i, c, val, qp, pp, qq);
                }
                if (a.mode == kLanczos) {
                    qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
                    if (lane == 0) {
                        red[(wl * TP + cl) * 3 + 0] = qp;
                        red[(wl * TP + cl) * 3 + 1] = pp;
                        red[(wl * TP + cl) * 3 + 2] = qq;
                    }
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (a.mode == kLanczos) {
        const int ncol = min(TP, a.T - c0);
        for (int cl = tid; cl < ncol; cl += blockDim.x) {
            double* dst = a.partials + ((int64_t)tile * a.T + c0 + cl) * 3;
#pragma unroll
            for (int k = 0; k < 3; ++k)
                dst[k] = red[(0 * TP + cl) * 3 + k] + red[(1 * TP + cl) * 3 + k] + red[(2 * TP + cl) * 3 + k] +
                         red[(3 * TP + cl) * 3 + k];
        }
    }
    if (tid == 0 && *serr) atomicExch(p.err, 1);
    if (warp == 0) tc::tmem_dealloc(tmem, NCOLS);
}

template <int KT, int TP, bool HALF>
cudaError_t launch_tp(const TcPoints& p, const MvmArgs<float>& a, int c0, cudaStream_t st) {
    constexpr int smem = tc_smem_bytes<TP>();
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(mvm_tc_kernel<KT, TP, HALF>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    mvm_tc_kernel<KT, TP, HALF><<<(unsigned)(a.Npad / kTcBM), 384, smem, st>>>(p, a, c0);
    return cudaGetLastError();
}

template <int KT, bool HALF>
cudaError_t launch_kt_half(const TcPoints& p, const MvmArgs<float>& a, int tpg, int c0, cudaStream_t st) {
    switch (tpg) {
        case 32: return launch_tp<KT, 32, HALF>(p, a, c0, st);
        case 64: return launch_tp<KT, 64, HALF>(p, a, c0, st);
        case 128: return launch_tp<KT, 128, HALF>(p, a, c0, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool tc_supported(int precision, int d) {
    return (precision == CIQ_PREC_BF16 || precision == CIQ_PREC_FP16) && d >= 1 && d <= 14;
}

// Columns of V per MVM launch group (T > 128 runs as groups of 128; the
// TMEM loads and stores move 32 columns, so a group is at least 32 wide).
int tc_group_t(int T) {
    if (T <= 32) return 32;
    if (T <= 64) return 64;
    return 128;
}

int tc_padded_t(int T) {
    if (T < 1 || T > 1024) return -1;
    const int g = tc_group_t(T);
    return (T + g - 1) / g * g;
}

int64_t tc_row_tiles(int64_t Npad) { return Npad / kTcBM; }

size_t tc_points_bytes(int64_t Npad, int T) {
    const int TP = tc_padded_t(T);
    if (TP < 0) return 0;
    const size_t pts = (size_t)Npad * kTcRowBytes;
    const size_t vb = (size_t)(Npad / kTcBN) * 2 * TP * 128;
    return 2 * pts + vb + 256 * 4 + (size_t)TP * sizeof(float) + 16 * sizeof(double) + 256;
}

TcPoints tc_points_layout(char* base, int64_t Npad, int T, int precision) {
    TcPoints p;
    p.Npad = Npad;
    p.TP = tc_padded_t(T);
    p.half = precision == CIQ_PREC_FP16 ? 1 : 0;
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
    return p;
}

cudaError_t launch_tc_prepare(const TcPoints& p, const float* Xp, int64_t N, int dp, int d, int kt,
                              cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(p.mean, 0, 16 * sizeof(double), st);
    if (e != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(p.err, 0, sizeof(int), st)) != cudaSuccess) return e;
    tc_mean_kernel<<<148, 256, 0, st>>>(Xp, N, dp, p.mean);
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

cudaError_t launch_mvm_tc(const TcPoints& p, const MvmArgs<float>& a, bool unit_columns, cudaStream_t st) {
    if (p.TP < 0 || a.T > p.TP || a.Npad != p.Npad || a.ldv != a.Npad) return cudaErrorInvalidValue;
    const float unit_scale = ldexpf(1.f, (int)floor(0.5 * log2((double)a.N)));
    tc_vscale_kernel<<<p.TP, 256, 0, st>>>(a.V, a.ldv, a.N, a.T, p.TP, unit_scale, unit_columns ? 1 : 0, p.vscale);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t work = (a.Npad / 8) * p.TP;
    if (p.half)
        tc_split_v_kernel<true><<<(unsigned)((work + 255) / 256), 256, 0, st>>>(a.V, a.ldv, a.T, p.TP,
                                                                                 tc_group_t(a.T), a.Npad,
                                                                                 p.vscale, p.vblk);
    else
        tc_split_v_kernel<false><<<(unsigned)((work + 255) / 256), 256, 0, st>>>(a.V, a.ldv, a.T, p.TP,
                                                                                  tc_group_t(a.T), a.Npad,
                                                                                  p.vscale, p.vblk);
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

}  // namespace ciq
