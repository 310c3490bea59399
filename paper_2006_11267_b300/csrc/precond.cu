// Pivoted-Cholesky preconditioner of msMINRES-CIQ (App. "Preconditioning
// msMINRES-CIQ"): the factor, its orthonormal basis and the FP32 applications
// of P^{+-1/2}.  See precond.cuh for the formulas.
//
//  * pc_cholesky_step: one greedy step of the partial pivoted Cholesky of
//    K_XX (Harbrecht, Peters and Schneider 2012): the pivot's kernel column,
//    minus the previous columns (float-pair dot), divided by the root of the
//    pivot's residual diagonal; the residual diagonal (FP64) is updated and
//    the next pivot (largest residual, first index on ties) is chosen by the
//    last block to finish.  One launch per column.
//  * gram_part / gram_reduce: G = L^T L with exact FP32 products summed as
//    float pairs within a row chunk and in FP64 across chunks.
//  * basis_from_factor: Qh = L W with W = U diag(s)^{-1/2} (FP64 accumulation).
//  * pc_reduce / pc_coef: C = diag(g) Qh^T X, a 64 x 64 register-tiled product
//    over row chunks (FP32 within a chunk, float pairs across chunks).
//  * pc_expand: out = sigma^{+-1} X + Qh C over 128-row tiles, with the
//    Lanczos epilogue (p = O - beta q_prev; q.p, p.p, q.q per tile as float
//    pairs of exact products, stored as FP64) for the preconditioned MVM.
#include <climits>

#include <algorithm>

#include "precond.cuh"

namespace ciq {

namespace {

constexpr int kRedRT = 128;     // r (basis column) tile of the reduction
constexpr int kRedTT = 64;      // t (right-hand side) tile
constexpr int kRedSub = 32;     // rows per shared-memory stage

int64_t chunk_rows(int64_t Npad, int R, int T) {
    // Row chunks for one wave of three blocks per SM (148 SMs), each chunk at
    // least 256 rows.
    const int64_t tiles = (int64_t)((R + kRedRT - 1) / kRedRT) * ((T + kRedTT - 1) / kRedTT);
    int64_t ch = std::max<int64_t>(1, 444 / tiles);
    ch = std::min<int64_t>(ch, std::max<int64_t>(1, Npad / 256));
    return round_up((Npad + ch - 1) / ch, kRedSub);
}

// Float pairs (hi + lo, about twice FP32's precision): FP64 runs at about
// 1/64 of FP32's rate on this part, and the Lanczos sums of the epilogue
// would otherwise dominate it.  Intrinsics keep every operation rounded as
// written (no contraction into FMAs).
struct FPair {
    float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ void pair_add(FPair& a, float x) {
    const float s = __fadd_rn(a.hi, x);
    const float bp = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bp)), __fsub_rn(x, bp));
    a.hi = s;
    a.lo = __fadd_rn(a.lo, err);
}

// a += x * y with the product's rounding error kept (FMA), so the pair holds
// the exact product sum to about 2^-48 relative.
__device__ __forceinline__ void pair_fma(FPair& a, float x, float y) {
    const float p = __fmul_rn(x, y);
    const float e = __fmaf_rn(x, y, -p);
    pair_add(a, p);
    a.lo = __fadd_rn(a.lo, e);
}

__device__ __forceinline__ FPair pair_warp_sum(FPair a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float h = __shfl_xor_sync(0xffffffffu, a.hi, o);
        const float l = __shfl_xor_sync(0xffffffffu, a.lo, o);
        pair_add(a, h);
        a.lo = __fadd_rn(a.lo, l);
    }
    return a;
}

// cpart[chunk][t][r] = sum over the chunk's rows of Qh[r][i] X[t][i].  A block
// takes a 128 (r) x 64 (t) tile of one row chunk with 128 threads, each an
// 8 x 8 register tile (64 FMAs per 16 floats read from shared memory); the
// next 32-row stage is loaded into registers while the current one is
// multiplied.
__global__ void __launch_bounds__(128, 3) pc_reduce(PrecondState pc, const float* X, int64_t ldx, int T,
                                                    int64_t rows_per_chunk, const int* stop) {
    if (stop && *stop) return;
    constexpr int LA = kRedRT + 4, LB = kRedTT + 4;        // padded rows (16-byte aligned)
    __shared__ __align__(16) float As[kRedSub][LA];
    __shared__ __align__(16) float Bs[kRedSub][LB];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3;
    const int r0 = blockIdx.x * kRedRT, t0 = blockIdx.y * kRedTT;
    const int64_t i_begin = (int64_t)blockIdx.z * rows_per_chunk;
    const int64_t i_end = min(i_begin + rows_per_chunk, pc.Npad);
    float acc[8][8] = {};
    // Per stage: 128 r x 32 rows of Qh (8 float4 per thread, 8 threads per
    // 128-byte row segment) and 64 t x 32 rows of X (4 float4 per thread).
    float4 na[8], nb[4];
    auto load = [&](int64_t i0) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 7, rr = e >> 3;
            const int r = r0 + rr;
            const int64_t i = i0 + 4 * q4;                  // i_end and Npad are multiples of 4
            na[m] = (r < pc.rank && i < i_end) ? *reinterpret_cast<const float4*>(pc.Qh + (int64_t)r * pc.Npad + i)
                                               : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 7, tt = e >> 3;
            const int t = t0 + tt;
            const int64_t i = i0 + 4 * q4;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < T && i < i_end) {
                const float* src = X + (int64_t)t * ldx + i;
                v.x = i < pc.N ? src[0] : 0.f;
                v.y = i + 1 < pc.N ? src[1] : 0.f;
                v.z = i + 2 < pc.N ? src[2] : 0.f;
                v.w = i + 3 < pc.N ? src[3] : 0.f;
            }
            nb[m] = v;
        }
    };
    if (i_begin < i_end) load(i_begin);
    for (int64_t i0 = i_begin; i0 < i_end; i0 += kRedSub) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 7, rr = e >> 3;
            As[4 * q4][rr] = na[m].x;
            As[4 * q4 + 1][rr] = na[m].y;
            As[4 * q4 + 2][rr] = na[m].z;
            As[4 * q4 + 3][rr] = na[m].w;
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 7, tt = e >> 3;
            Bs[4 * q4][tt] = nb[m].x;
            Bs[4 * q4 + 1][tt] = nb[m].y;
            Bs[4 * q4 + 2][tt] = nb[m].z;
            Bs[4 * q4 + 3][tt] = nb[m].w;
        }
        __syncthreads();
        if (i0 + kRedSub < i_end) load(i0 + kRedSub);
#pragma unroll 4
        for (int ii = 0; ii < kRedSub; ++ii) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[ii][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[ii][ty * 8 + 4]);
            const float4 b0 = *reinterpret_cast<const float4*>(&Bs[ii][tx * 8]);
            const float4 b1 = *reinterpret_cast<const float4*>(&Bs[ii][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], bv[v], acc[u][v]);
        }
        __syncthreads();
    }
    float* dst = pc.cpart + (int64_t)blockIdx.z * pc.rank * T;      // [chunk][t][r]
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int t = t0 + tx * 8 + v;
        if (t >= T) break;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int r = r0 + ty * 8 + u;
            if (r < pc.rank) dst[(int64_t)t * pc.rank + r] = acc[u][v];
        }
    }
}

__global__ void __launch_bounds__(256) pc_coef(PrecondState pc, int T, int nchunks, bool inverse_root,
                                               float* vscale, int TP, const int* stop) {
    if (stop && *stop) return;
    const int t = blockIdx.x;
    double nrm2 = 0.0;
    const double is = 1.0 / (double)pc.sigma;
    for (int r = threadIdx.x; r < pc.rank; r += blockDim.x) {
        FPair acc;
        for (int c = 0; c < nchunks; ++c) pair_add(acc, pc.cpart[((int64_t)c * T + t) * pc.rank + r]);
        const double s = (double)acc.hi + (double)acc.lo;
        const double g = (double)(inverse_root ? pc.gm[r] : pc.gp[r]);
        pc.coef[(int64_t)r * T + t] = (float)(s * g);
        nrm2 += (g * g + 2.0 * g * is) * s * s;
    }
    if (!vscale) return;
    __shared__ double red[8];
    nrm2 = warp_sum(nrm2);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = nrm2;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = is * is;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        const double nrm = sqrt(fmax(s, 0.0));
        vscale[t] = nrm > 0.0 ? ldexpf(1.f, (int)floor(log2(sqrt((double)pc.N) / nrm))) : 1.f;
        if (t == 0)
            for (int c = T; c < TP; ++c) vscale[c] = ldexpf(1.f, (int)floor(0.5 * log2((double)pc.N)));
    }
}

// The operand scale of U = v / sigma when P has no low-rank part.
__global__ void pc_unit_scale(PrecondState pc, int T, int TP, float* vscale, const int* stop) {
    if (stop && *stop) return;
    for (int c = threadIdx.x; c < TP; c += blockDim.x) {
        const double nrm = c < T ? 1.0 / (double)pc.sigma : 1.0;
        vscale[c] = ldexpf(1.f, (int)floor(log2(sqrt((double)pc.N) / nrm)));
    }
}

// out[t][i] = alpha X[t][i] + sum_r Qh[r][i] coef[r][t] over a 128-row tile
// and 64 columns; LANCZOS: p = out - beta_t qprev[t][i] with partial sums.
template <bool LANCZOS>
__global__ void __launch_bounds__(128, 3) pc_expand(PrecondState pc, const float* X, int64_t ldx, int T, float alpha,
                                                 float* out, int64_t ldo, const float* q, float* qprev,
                                                 float* pout, const double* beta, double* partials,
                                                 const int* stop) {
    // A 128-row x 64-column tile of alpha X + Qh C with 128 threads, each 8
    // rows x 8 columns (64 FMAs per 16 floats read from shared memory); the
    // next 32 basis columns are loaded into registers while the current ones
    // are multiplied.
    if (stop && *stop) return;
    constexpr int RT = 32;
    __shared__ __align__(16) float Qs[RT][128];
    __shared__ __align__(16) float Cs[RT][64];
    __shared__ double red[4][8][3];
    const int tid = threadIdx.x, tx = tid & 7, ty = tid >> 3, lane = tid & 31, warp = tid >> 5;
    const int64_t i0 = (int64_t)blockIdx.x * 128;
    const int t0 = blockIdx.y * 64;
    float acc[8][8] = {};
    float4 nq[8], nc[4];
    auto load = [&](int r0) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 31, rr = e >> 5;
            const int r = r0 + rr;
            nq[m] = r < pc.rank ? *reinterpret_cast<const float4*>(pc.Qh + (int64_t)r * pc.Npad + i0 + 4 * q4)
                                : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = tid + 128 * m;
            const int q4 = e & 15, rr = e >> 4;
            const int r = r0 + rr;
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (r < pc.rank) {
                const float* src = pc.coef + (int64_t)r * T + t0 + 4 * q4;
                const int tb = t0 + 4 * q4;
                v.x = tb < T ? src[0] : 0.f;
                v.y = tb + 1 < T ? src[1] : 0.f;
                v.z = tb + 2 < T ? src[2] : 0.f;
                v.w = tb + 3 < T ? src[3] : 0.f;
            }
            nc[m] = v;
        }
    };
    if (pc.rank > 0) load(0);
    for (int r0 = 0; r0 < pc.rank; r0 += RT) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int e = tid + 128 * m;
            *reinterpret_cast<float4*>(&Qs[e >> 5][4 * (e & 31)]) = nq[m];
        }
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            const int e = tid + 128 * m;
            *reinterpret_cast<float4*>(&Cs[e >> 4][4 * (e & 15)]) = nc[m];
        }
        __syncthreads();
        if (r0 + RT < pc.rank) load(r0 + RT);
#pragma unroll 4
        for (int rr = 0; rr < RT; ++rr) {
            const float4 a0 = *reinterpret_cast<const float4*>(&Qs[rr][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&Qs[rr][ty * 8 + 4]);
            const float4 c0 = *reinterpret_cast<const float4*>(&Cs[rr][tx * 8]);
            const float4 c1 = *reinterpret_cast<const float4*>(&Cs[rr][tx * 8 + 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float cv[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
#pragma unroll
            for (int u = 0; u < 8; ++u)
#pragma unroll
                for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(av[u], cv[v], acc[u][v]);
        }
        __syncthreads();
    }
    // Thread (tx, ty) holds rows i0 + 8 ty + u and columns t0 + 8 tx + v.
#pragma unroll
    for (int v = 0; v < 8; ++v) {
        const int t = t0 + tx * 8 + v;
        const bool col = t < T;
        FPair qp, pp, qq;
        if (col) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int64_t i = i0 + ty * 8 + u;
                const float x = i < pc.N ? X[(int64_t)t * ldx + i] : 0.f;
                const float o = fmaf(alpha, x, acc[u][v]);
                if (!LANCZOS) {
                    if (i < pc.N) out[(int64_t)t * ldo + i] = o;
                    else if (ldo >= pc.Npad) out[(int64_t)t * ldo + i] = 0.f;
                } else {
                    const int64_t idx = (int64_t)t * pc.Npad + i;
                    const float p = i < pc.N ? o - (float)beta[t] * qprev[idx] : 0.f;
                    (pout ? pout : qprev)[idx] = p;
                    const float qv = q[idx];
                    pair_fma(qp, qv, p);
                    pair_fma(pp, p, p);
                    pair_fma(qq, qv, qv);
                }
            }
        }
        if (LANCZOS) {
            // The 4 threads of a warp with this tx (lanes tx, tx + 8, ...), then the 4 warps.
#pragma unroll
            for (int o = 8; o < 32; o <<= 1) {
                FPair* ps[3] = {&qp, &pp, &qq};
#pragma unroll
                for (int k = 0; k < 3; ++k) {
                    const float h = __shfl_xor_sync(0xffffffffu, ps[k]->hi, o);
                    const float l = __shfl_xor_sync(0xffffffffu, ps[k]->lo, o);
                    pair_add(*ps[k], h);
                    ps[k]->lo = __fadd_rn(ps[k]->lo, l);
                }
            }
            if (lane < 8) {
                red[warp][lane][0] = (double)qp.hi + (double)qp.lo;
                red[warp][lane][1] = (double)pp.hi + (double)pp.lo;
                red[warp][lane][2] = (double)qq.hi + (double)qq.lo;
            }
            __syncthreads();
            if (tid < 8 && t0 + tid * 8 + v < T) {
                const int tc = t0 + tid * 8 + v;
                double* dst = partials + ((int64_t)blockIdx.x * T + tc) * 3;
#pragma unroll
                for (int k = 0; k < 3; ++k) dst[k] = red[0][tid][k] + red[1][tid][k] + red[2][tid][k] + red[3][tid][k];
            }
            __syncthreads();
        }
    }
}

// ---------------------------------------------------------------- setup ----
struct CholWork {
    int* ispiv;          // [Npad]
    double* dmax;        // [rank + 1] residual diagonal of each pivot when chosen
    double* bval;        // [blocks]
    int* bidx;           // [blocks]
    unsigned* counter;
};

CholWork chol_work(void* base, int64_t Npad) {
    CholWork w;
    char* p = static_cast<char*>(base);
    const int64_t blocks = Npad / 256 + 1;
    w.ispiv = reinterpret_cast<int*>(p);
    p += round_up(Npad * sizeof(int), 256);
    w.dmax = reinterpret_cast<double*>(p);
    p += round_up((kPcMaxRank + 1) * sizeof(double), 256);
    w.bval = reinterpret_cast<double*>(p);
    p += round_up(blocks * sizeof(double), 256);
    w.bidx = reinterpret_cast<int*>(p);
    p += round_up(blocks * sizeof(int), 256);
    w.counter = reinterpret_cast<unsigned*>(p);
    return w;
}

__global__ void pc_cholesky_init(int64_t N, int64_t Npad, double s, double* dres, CholWork w, int* piv,
                                 int* rank_out, int rank, const float* Ct, int rk) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < Npad) {
        double d = i < N ? s : -1.0;
        if (i < N && rk > 0) {
            // Diagonal of K - C C^T: s - |c_i|^2 (float pair of exact squares).
            FPair c2;
            for (int k = 0; k < rk; ++k) {
                const float c = Ct[(int64_t)k * Npad + i];
                pair_fma(c2, c, c);
            }
            d = s - ((double)c2.hi + (double)c2.lo);
        }
        dres[i] = d;
        w.ispiv[i] = 0;
    }
    if (i == 0) {
        piv[0] = 0;                   // every diagonal entry of K_XX is s: the first index wins
        w.dmax[0] = s;
        *w.counter = 0u;
        *rank_out = rank;
    }
}

// First pivot of K - C C^T: the largest residual diagonal entry (smallest
// index on ties), one block.
__global__ void __launch_bounds__(1024) pc_cholesky_first(int64_t N, const double* dres, CholWork w, int* piv) {
    __shared__ double rv[32];
    __shared__ int ri[32];
    double bv = -2.0;
    int bi = INT_MAX;
    for (int64_t i = threadIdx.x; i < N; i += 1024)
        if (dres[i] > bv) { bv = dres[i]; bi = (int)i; }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((threadIdx.x & 31) == 0) { rv[threadIdx.x >> 5] = bv; ri[threadIdx.x >> 5] = bi; }
    __syncthreads();
    if (threadIdx.x == 0) {
        bv = rv[0];
        bi = ri[0];
        for (int q = 1; q < 32; ++q)
            if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) { bv = rv[q]; bi = ri[q]; }
        piv[0] = bi == INT_MAX ? 0 : bi;
        w.dmax[0] = bv;
    }
}

template <int KT>
__global__ void __launch_bounds__(256) pc_cholesky_step(const float* Xp, int64_t N, int64_t Npad, int dp, float s,
                                                        int k, float* L, int* piv, double* dres, CholWork w,
                                                        int* rank_out, const float* Ct, int rk) {
    __shared__ float Lp[kPcMaxRank];
    __shared__ float Cp[kPcMaxTrain];
    __shared__ float xp[kMaxDimPad];
    __shared__ double rv[8];
    __shared__ int ri[8];
    __shared__ bool last;
    const double dpiv = w.dmax[k];
    if (!(dpiv > 0.0)) {                       // residual exhausted: the factor has k columns
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            atomicMin(rank_out, k);
            w.dmax[k + 1] = 0.0;               // and every later step returns here too
        }
        return;
    }
    const int ip = piv[k];
    const int tid = threadIdx.x;
    for (int m = tid; m < k; m += 256) Lp[m] = L[(int64_t)m * Npad + ip];
    for (int m = tid; m < rk; m += 256) Cp[m] = Ct[(int64_t)m * Npad + ip];
    if (tid < dp) xp[tid] = Xp[(int64_t)ip * dp + tid];
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * 256 + tid;
    double dnew = -1.0;
    if (i < N) {
        float r2 = 0.f;
        for (int c = 0; c < dp; ++c) {
            const float df = Xp[i * dp + c] - xp[c];
            r2 = fmaf(df, df, r2);
        }
        // The kernel value minus the earlier columns' contributions, summed as
        // a float pair of exact products (FP64 is slow here; see FPair).
        // With a low-rank term, the column of K - C C^T: c_i . c_p joins the dot.
        FPair dot;
        for (int m = 0; m < k; ++m) pair_fma(dot, L[(int64_t)m * Npad + i], Lp[m]);
        for (int m = 0; m < rk; ++m) pair_fma(dot, Ct[(int64_t)m * Npad + i], Cp[m]);
        double col = (double)kernel_value<KT>(r2, s) - ((double)dot.hi + (double)dot.lo);
        const bool was_pivot = w.ispiv[i] != 0;
        if (was_pivot) col = 0.0;              // earlier pivot rows of the Schur complement are 0
        const float l = (float)(col / sqrt(dpiv));
        L[(int64_t)k * Npad + i] = l;
        if (was_pivot || i == ip) {
            dnew = 0.0;
            if (i == ip) w.ispiv[i] = 1;
        } else {
            dnew = dres[i] - (double)l * (double)l;
        }
        dres[i] = dnew;
    } else if (i < Npad) {
        L[(int64_t)k * Npad + i] = 0.f;
    }
    // Block argmax (largest value, then smallest index).
    double bv = dnew;
    int bi = i < N ? (int)i : INT_MAX;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    if ((tid & 31) == 0) { rv[tid >> 5] = bv; ri[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
        bv = rv[0];
        bi = ri[0];
        for (int q = 1; q < 8; ++q)
            if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) { bv = rv[q]; bi = ri[q]; }
        w.bval[blockIdx.x] = bv;
        w.bidx[blockIdx.x] = bi;
        __threadfence();
        last = atomicAdd(w.counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    // Last block: argmax over the blocks, the next pivot.
    __threadfence();
    bv = -2.0;
    bi = INT_MAX;
    for (int b = tid; b < (int)gridDim.x; b += 256) {
        const double ov = ((volatile double*)w.bval)[b];
        const int oi = ((volatile int*)w.bidx)[b];
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
    }
    __syncthreads();
    if ((tid & 31) == 0) { rv[tid >> 5] = bv; ri[tid >> 5] = bi; }
    __syncthreads();
    if (tid == 0) {
        bv = rv[0];
        bi = ri[0];
        for (int q = 1; q < 8; ++q)
            if (rv[q] > bv || (rv[q] == bv && ri[q] < bi)) { bv = rv[q]; bi = ri[q]; }
        piv[k + 1] = bi == INT_MAX ? 0 : bi;
        w.dmax[k + 1] = bv;
        *w.counter = 0u;
    }
}

// gpart[chunk][a][b] = sum over the chunk's rows of L[a][i] L[b][i] (32 x 32
// tiles with a-tile <= b-tile).
__global__ void __launch_bounds__(256) gram_part(const float* L, int64_t Npad, int R, int64_t rows_per_chunk,
                                                 double* gpart) {
    if (blockIdx.x > blockIdx.y) return;
    __shared__ float As[64][33];
    __shared__ float Bs[64][33];
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int a0 = blockIdx.x * 32, b0 = blockIdx.y * 32;
    const int64_t i_begin = (int64_t)blockIdx.z * rows_per_chunk;
    const int64_t i_end = min(i_begin + rows_per_chunk, Npad);
    // Float-pair accumulation of exact products (the product's error from an
    // FMA, Knuth's 2Sum for the sum; intrinsics, so nothing is contracted):
    // about twice FP32's precision at the FP32 pipe's rate.
    float hi[2][2] = {}, lo[2][2] = {};
    for (int64_t i0 = i_begin; i0 < i_end; i0 += 64) {
        for (int e = tid; e < 64 * 32; e += 256) {
            const int ii = e & 63, cc = e >> 6;
            const int64_t i = i0 + ii;
            As[ii][cc] = (a0 + cc < R && i < i_end) ? L[(int64_t)(a0 + cc) * Npad + i] : 0.f;
            Bs[ii][cc] = (b0 + cc < R && i < i_end) ? L[(int64_t)(b0 + cc) * Npad + i] : 0.f;
        }
        __syncthreads();
        for (int ii = 0; ii < 64; ++ii) {
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int v = 0; v < 2; ++v) {
                    const float x = As[ii][ty * 2 + u], y = Bs[ii][tx * 2 + v];
                    const float p = __fmul_rn(x, y);
                    const float pe = __fmaf_rn(x, y, -p);
                    const float s = __fadd_rn(hi[u][v], p);
                    const float bp = __fsub_rn(s, hi[u][v]);
                    const float err = __fadd_rn(__fsub_rn(hi[u][v], __fsub_rn(s, bp)), __fsub_rn(p, bp));
                    hi[u][v] = s;
                    lo[u][v] = __fadd_rn(lo[u][v], __fadd_rn(err, pe));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 2; ++v) {
            const int a = a0 + ty * 2 + u, b = b0 + tx * 2 + v;
            if (a < R && b < R) gpart[((int64_t)blockIdx.z * R + a) * R + b] = (double)hi[u][v] + (double)lo[u][v];
        }
}

__global__ void gram_reduce(const double* gpart, int R, int nchunks, double* G) {
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (int64_t)R * R) return;
    const int a = (int)(e / R), b = (int)(e % R);
    if (a / 32 > b / 32) return;                 // written from the transposed entry
    double s = 0.0;
    for (int c = 0; c < nchunks; ++c) s += gpart[((int64_t)c * R + a) * R + b];
    G[a + (int64_t)b * R] = s;
    G[b + (int64_t)a * R] = s;
}

// Qh[c][i] = sum_m L[m][i] W[m][c], 32 columns per block, one row per thread.
template <typename TIn>
__global__ void __launch_bounds__(128) basis_from_factor(const TIn* L, int64_t Npad, int R, const double* W,
                                                         int Rk, float* Qh) {
    __shared__ double Ws[32][32];
    const int64_t i = (int64_t)blockIdx.x * 128 + threadIdx.x;
    const int c0 = blockIdx.y * 32;
    double acc[32];
#pragma unroll
    for (int c = 0; c < 32; ++c) acc[c] = 0.0;
    for (int m0 = 0; m0 < R; m0 += 32) {
        for (int e = threadIdx.x; e < 32 * 32; e += 128) {
            const int mm = e >> 5, cc = e & 31;
            Ws[mm][cc] = (m0 + mm < R && c0 + cc < Rk) ? W[(m0 + mm) + (int64_t)(c0 + cc) * R] : 0.0;
        }
        __syncthreads();
        const int mend = min(32, R - m0);
        for (int mm = 0; mm < mend; ++mm) {
            const double l = (double)L[(int64_t)(m0 + mm) * Npad + i];
#pragma unroll
            for (int c = 0; c < 32; ++c) acc[c] = fma(l, Ws[mm][c], acc[c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int c = 0; c < 32; ++c)
        if (c0 + c < Rk) Qh[(int64_t)(c0 + c) * Npad + i] = (float)acc[c];
}

}  // namespace

int64_t pc_chunks(int64_t Npad) {
    // Worst case over rank and T (chunk_rows is at least kRedSub rows).
    return (Npad + kRedSub - 1) / kRedSub;
}

size_t pc_scratch_floats(int64_t Npad, int rank, int T) {
    // Partial sums for the most row chunks any rank up to `rank` uses (the
    // chunk count only falls as the rank needs more tiles, so rank 1 has the
    // most), then the coefficients.
    const int64_t rows = chunk_rows(Npad, 1, T);
    const int64_t nch = (Npad + rows - 1) / rows;
    return (size_t)nch * rank * T + (size_t)rank * T;
}

cudaError_t launch_pc_apply(const PrecondState& pc, const float* X, int64_t ldx, int T, bool inverse_root,
                            float* out, int64_t ldo, const int* stop, cudaStream_t st, float* vscale, int TP) {
    if (pc.rank > 0) {
        const int64_t rows = chunk_rows(pc.Npad, pc.rank, T);
        const int nch = (int)((pc.Npad + rows - 1) / rows);
        dim3 g1((pc.rank + kRedRT - 1) / kRedRT, (T + kRedTT - 1) / kRedTT, nch);
        pc_reduce<<<g1, 128, 0, st>>>(pc, X, ldx, T, rows, stop);
        pc_coef<<<T, 256, 0, st>>>(pc, T, nch, inverse_root, vscale, TP, stop);
    } else if (vscale) {
        pc_unit_scale<<<1, 256, 0, st>>>(pc, T, TP, vscale, stop);
    }
    dim3 g2((unsigned)(pc.Npad / 128), (T + 63) / 64);
    pc_expand<false><<<g2, 128, 0, st>>>(pc, X, ldx, T, inverse_root ? pc.inv_sigma : pc.sigma, out, ldo, nullptr,
                                         nullptr, nullptr, nullptr, nullptr, stop);
    return cudaGetLastError();
}

cudaError_t launch_pc_lanczos(const PrecondState& pc, const float* Oraw, const float* q, float* qprev, float* pout,
                              const double* beta, double* partials, int T, const int* stop, cudaStream_t st) {
    if (pc.rank > 0) {
        const int64_t rows = chunk_rows(pc.Npad, pc.rank, T);
        const int nch = (int)((pc.Npad + rows - 1) / rows);
        dim3 g1((pc.rank + kRedRT - 1) / kRedRT, (T + kRedTT - 1) / kRedTT, nch);
        pc_reduce<<<g1, 128, 0, st>>>(pc, Oraw, pc.Npad, T, rows, stop);
        pc_coef<<<T, 256, 0, st>>>(pc, T, nch, true, nullptr, 0, stop);
    }
    dim3 g2((unsigned)(pc.Npad / 128), (T + 63) / 64);
    pc_expand<true><<<g2, 128, 0, st>>>(pc, Oraw, pc.Npad, T, pc.inv_sigma, nullptr, 0, q, qprev, pout, beta,
                                        partials, stop);
    return cudaGetLastError();
}

size_t pc_cholesky_work_bytes(int64_t Npad) {
    const int64_t blocks = Npad / 256 + 1;
    return round_up(Npad * sizeof(int), 256) + round_up((kPcMaxRank + 1) * sizeof(double), 256) +
           round_up(blocks * sizeof(double), 256) + round_up(blocks * sizeof(int), 256) + 256;
}

cudaError_t launch_pivoted_cholesky(const float* Xp, int64_t N, int64_t Npad, int dp, int kt, float outputscale,
                                    int rank, float* L, int* piv, double* dres, void* work, int* rank_out,
                                    cudaStream_t st, const float* Ct, int rk) {
    if (rank < 1 || rank > kPcMaxRank || rk < 0 || rk > kPcMaxTrain || (rk > 0 && !Ct)) return cudaErrorInvalidValue;
    CholWork w = chol_work(work, Npad);
    cudaError_t e = cudaMemsetAsync(L, 0, sizeof(float) * (size_t)rank * Npad, st);
    if (e != cudaSuccess) return e;
    pc_cholesky_init<<<(unsigned)((Npad + 255) / 256), 256, 0, st>>>(N, Npad, (double)outputscale, dres, w, piv,
                                                                      rank_out, rank, Ct, rk);
    if (rk > 0) pc_cholesky_first<<<1, 1024, 0, st>>>(N, dres, w, piv);
    const unsigned blocks = (unsigned)((Npad + 255) / 256);
    for (int k = 0; k < rank; ++k) {
        if (kt == CIQ_RBF)
            pc_cholesky_step<CIQ_RBF><<<blocks, 256, 0, st>>>(Xp, N, Npad, dp, outputscale, k, L, piv, dres, w,
                                                               rank_out, Ct, rk);
        else
            pc_cholesky_step<CIQ_MATERN52><<<blocks, 256, 0, st>>>(Xp, N, Npad, dp, outputscale, k, L, piv, dres,
                                                                    w, rank_out, Ct, rk);
    }
    return cudaGetLastError();
}

int64_t pc_gram_scratch(int64_t Npad, int R) {
    const int64_t rows = 4096;
    const int64_t nch = (Npad + rows - 1) / rows;
    return nch * R * R;
}

cudaError_t launch_gram(const float* L, int64_t Npad, int R, double* gpart, double* G, cudaStream_t st) {
    const int64_t rows = 4096;
    const int nch = (int)((Npad + rows - 1) / rows);
    const int rt = (R + 31) / 32;
    gram_part<<<dim3(rt, rt, nch), 256, 0, st>>>(L, Npad, R, rows, gpart);
    const int64_t n = (int64_t)R * R;
    gram_reduce<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(gpart, R, nch, G);
    return cudaGetLastError();
}

cudaError_t launch_basis_from_factor(const float* L, int64_t Npad, int R, const double* W, int Rk, float* Qh,
                                     cudaStream_t st) {
    if (Rk < 1) return cudaSuccess;
    basis_from_factor<float><<<dim3((unsigned)(Npad / 128), (Rk + 31) / 32), 128, 0, st>>>(L, Npad, R, W, Rk, Qh);
    return cudaGetLastError();
}

cudaError_t launch_product_f64(const double* A, int64_t Npad, int R, const double* W, int Rk, float* out,
                               cudaStream_t st) {
    if (Rk < 1) return cudaSuccess;
    basis_from_factor<double><<<dim3((unsigned)(Npad / 128), (Rk + 31) / 32), 128, 0, st>>>(A, Npad, R, W, Rk, out);
    return cudaGetLastError();
}

cudaError_t launch_lowrank_apply(const PrecondState& lr, const float* V, float* O, int T, const int* stop,
                                  cudaStream_t st) {
    if (lr.rank <= 0) return cudaSuccess;
    const int64_t rows = chunk_rows(lr.Npad, lr.rank, T);
    const int nch = (int)((lr.Npad + rows - 1) / rows);
    dim3 g1((lr.rank + kRedRT - 1) / kRedRT, (T + kRedTT - 1) / kRedTT, nch);
    pc_reduce<<<g1, 128, 0, st>>>(lr, V, lr.Npad, T, rows, stop);
    pc_coef<<<T, 256, 0, st>>>(lr, T, nch, true, nullptr, 0, stop);
    dim3 g2((unsigned)(lr.Npad / 128), (T + 63) / 64);
    pc_expand<false><<<g2, 128, 0, st>>>(lr, O, lr.Npad, T, 1.f, O, lr.Npad, nullptr, nullptr, nullptr, nullptr,
                                         nullptr, stop);
    return cudaGetLastError();
}

cudaError_t launch_lowrank_lanczos(const PrecondState& pc, const float* V, const float* Oraw, const float* q,
                                   float* qprev, float* pout, const double* beta, double* partials, int T,
                                   const int* stop, cudaStream_t st) {
    if (pc.rank > 0) {
        const int64_t rows = chunk_rows(pc.Npad, pc.rank, T);
        const int nch = (int)((pc.Npad + rows - 1) / rows);
        dim3 g1((pc.rank + kRedRT - 1) / kRedRT, (T + kRedTT - 1) / kRedTT, nch);
        pc_reduce<<<g1, 128, 0, st>>>(pc, V, pc.Npad, T, rows, stop);
        pc_coef<<<T, 256, 0, st>>>(pc, T, nch, true, nullptr, 0, stop);
    }
    dim3 g2((unsigned)(pc.Npad / 128), (T + 63) / 64);
    pc_expand<true><<<g2, 128, 0, st>>>(pc, Oraw, pc.Npad, T, 1.f, nullptr, 0, q, qprev, pout, beta, partials, stop);
    return cudaGetLastError();
}

}  // namespace ciq
