// Batched msMINRES-CIQ kernels: many independent problems of uneven N, d and
// kernel, each with its own right-hand sides, advanced together.
//
// Every phase of Algorithm "ciq" (points, pre-pass, initialisation, J x
// (kernel MVM + msMINRES step), combination, summary) runs as ONE launch over
// all problems that still need it, instead of one launch per problem: block b
// takes work item b of a device work list (DevList), finds its problem by a
// binary search over the list's item prefix, and runs the same device body as
// the single-problem kernel of that phase with the block coordinates of that
// item.  The per-problem arithmetic is therefore identical to the
// single-problem path, bit for bit.
//
// The MVM is the only phase whose code depends on the problem (kernel type
// and padded dimension are template parameters of its body), so it launches
// once per class present, over that class's list.  Between batches of
// iterations, rebuild_lists drops every problem whose columns have all
// stopped, so the later, shorter launches carry only live work.
#include "batched.cuh"
#include "krylov_body.cuh"
#include "mvm_simt_body.cuh"

namespace ciq {

namespace {

__global__ void __launch_bounds__(256) batched_setup_kernel(const BatchProblem* probs, int phase, uint64_t seed,
                                                            int Q, DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const BatchProblem& bp = probs[p];
    switch (phase) {
        case kBatchPrepare: {
            const MvmArgs<float>& m = bp.mvm[0];
            const int64_t e = (int64_t)local * 256 + threadIdx.x;
            if (e >= m.Npad * m.dp) return;
            const int64_t i = e / m.dp;
            const int k = (int)(e % m.dp);
            bp.Xp[e] = (i < m.N && k < bp.d) ? (float)((double)bp.X[i * bp.d + k] * bp.inv_ls) : 0.f;
            return;
        }
        case kBatchReset: {
            const KrylovState<float>& s = bp.ks;
            for (int i = threadIdx.x; i < s.jmax + 2; i += blockDim.x) s.cnt[i] = 0;
            if (threadIdx.x == 0) *s.all_done = 0;
            return;
        }
        case kBatchInitRhs: {
            const KrylovState<float> s = bp.ks;
            init_rhs_body<float>(s, bp.B, local % s.nchunks, local / s.nchunks);
            return;
        }
        case kBatchInitState: {
            const KrylovState<float> s = bp.ks;
            init_state_body<float>(s, local % s.nchunks, local / s.nchunks);
            return;
        }
        case kBatchPreInitA: {
            const LanczosState<float> s = bp.ls;
            lanczos_init_a_body<float>(s, nullptr, seed, local, 0);
            return;
        }
        case kBatchPreInitB: {
            const LanczosState<float> s = bp.ls;
            lanczos_init_b_body<float>(s, local, 0);
            return;
        }
        case kBatchNodesGiven:
            if (threadIdx.x == 0) nodes_from_bounds_body(bp.nodes, Q, bp.lmin, bp.lmax);
            return;
        case kBatchCombine: {
            const KrylovState<float> s = bp.ks;
            const int nbx = (int)((s.N + 255) / 256);
            combine_body<float>(s, bp.out, local % nbx, local / nbx);
            return;
        }
        default:
            return;
    }
}

template <int KT, int TC, int DP, bool WIDE>
__global__ void __launch_bounds__(256) batched_mvm_kernel(const BatchProblem* probs, DevList L, int prepass,
                                                          int parity) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const BatchProblem& bp = probs[p];
    // The arguments live in shared memory, read where used (like kernel
    // parameters of the single-problem launch), not held in registers.
    __shared__ MvmArgs<float> a;
    if (threadIdx.x == 0) a = prepass ? bp.pre[parity] : bp.mvm[parity];
    const int tiles = prepass ? bp.pre_tiles : bp.mvm_tiles;
    __syncthreads();
    if constexpr (WIDE) {
        mvm_wide_body<KT, TC, DP>(a, local % tiles, local / tiles);
    } else {
        mvm_narrow_body<float, KT, TC, DP>(a, local % tiles, local / tiles);
    }
}

__global__ void __launch_bounds__(256) batched_lanczos_step_kernel(const BatchProblem* probs, int j, DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const LanczosState<float> s = probs[p].ls;
    lanczos_step_body<float>(s, j, local, 0);
}

__global__ void batched_bounds_nodes_kernel(const BatchProblem* probs, int Q, double lmax_margin, double lmin_div,
                                            DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const BatchProblem& bp = probs[p];
    const LanczosState<float> s = bp.ls;
    bounds_nodes_body<float>(s, bp.nodes, Q, bp.noise, lmax_margin, lmin_div, 0, 0);
}

__global__ void __launch_bounds__(256) batched_step_scalar_kernel(const BatchProblem* probs, int j, int final_pass,
                                                                  DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    step_scalar_body<float, false>(probs[p].ks, j, final_pass, local);
}

__global__ void __launch_bounds__(256, 3) batched_step_vector_kernel(const BatchProblem* probs, int j, DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const KrylovState<float> s = probs[p].ks;
    step_vector_body<float, false>(s, j, local % s.nchunks, local / s.nchunks);
}

// Largest eigenvalue of the symmetric tridiagonal (diag[0..J), off[1..J))
// by multisection over one warp: each round the 32 lanes take Sturm counts
// at 32 interior points of the bracket, which shrinks 33-fold, until it
// stops shrinking (FP64 resolution), about 11 rounds instead of the ~60
// serial bisection steps of tridiag_extreme (each step a pass of J FP64
// divisions; J reaches the solve's iteration count).
__device__ double tridiag_max_warp(const double* diag, const double* off, int J) {
    const int lane = threadIdx.x & 31;
    double lo = 1e300, hi = -1e300;
    for (int k = lane; k < J; k += 32) {
        const double r = (k > 0 ? fabs(off[k]) : 0.0) + (k + 1 < J ? fabs(off[k + 1]) : 0.0);
        lo = fmin(lo, diag[k] - r);
        hi = fmax(hi, diag[k] + r);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    for (int round = 0; round < 24; ++round) {
        const double x = lo + (hi - lo) * (double)(lane + 1) / 33.0;
        const unsigned above = __ballot_sync(0xffffffffu, sturm_count(diag, off, J, x) == J);
        const int first = above ? __ffs(above) - 1 : 32;        // first point above every eigenvalue
        const double nhi = __shfl_sync(0xffffffffu, x, first < 32 ? first : 31);
        const double nlo = __shfl_sync(0xffffffffu, x, first > 0 ? first - 1 : 0);
        const double new_hi = first < 32 ? nhi : hi;
        const double new_lo = first > 0 ? nlo : lo;
        if (!(new_hi < hi || new_lo > lo)) break;
        lo = new_lo;
        hi = new_hi;
    }
    return 0.5 * (lo + hi);
}

__global__ void batched_summary_kernel(const BatchProblem* probs, int final_j, double* packed, DevList L) {
    int p, local;
    if (!list_item(L, blockIdx.x, p, local)) return;
    const BatchProblem& bp = probs[p];
    const KrylovState<float> s = bp.ks;
    summary_body<float>(s, final_j, 0, 0);
    // The largest Ritz value of column 0's msMINRES tridiagonal (the
    // spectral check of learned bounds), by the whole warp.
    double th = 0.0;
    if (s.tri) {
        __syncwarp();
        const int J = s.iters[0];
        if (J >= 1) th = tridiag_max_warp(s.tri, s.tri + s.jmax + 1, J);
    }
    if (threadIdx.x != 0) return;
    double* dst = packed + (int64_t)p * kSummaryStride;
    for (int k = 0; k < 8; ++k) dst[k] = s.summary[k];
    for (int k = 0; k < kNodeCount; ++k) dst[8 + k] = bp.nodes[k];
    dst[8 + kNodeCount] = th;
    dst[9 + kNodeCount] = (bp.tcp.err && *bp.tcp.err) ? 1.0 : 0.0;
}

// Exclusive scan of one int per thread over a 1024-thread block; *total gets the sum.
__device__ __forceinline__ int block_exclusive_scan(int v, int* warp_tot, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int t = warp_tot[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += y;
        }
        warp_tot[lane] = t;               // inclusive over warps
    }
    __syncthreads();
    const int before = warp == 0 ? 0 : warp_tot[warp - 1];
    *total = warp_tot[31];
    return before + x - v;
}

// Block l rebuilds dynamic list l over the problems with list_items[l] > 0
// whose columns have not all stopped (*all_done == 0).
__global__ void __launch_bounds__(1024) rebuild_lists_kernel(const BatchProblem* probs, int P, const int* order,
                                                             DynLists lists, int* totals) {
    __shared__ int warp_tot[32];
    const int l = blockIdx.x;
    const DevList L = lists.l[l];
    const int per = (P + 1023) / 1024;
    const int p0 = min(P, (int)threadIdx.x * per), p1 = min(P, p0 + per);
    int n = 0, items = 0;
    for (int q = p0; q < p1; ++q) {
        const BatchProblem& bp = probs[order[q]];
        const int c = bp.list_items[l];
        if (c <= 0 || *bp.ks.all_done) continue;
        items += c;
        ++n;
    }
    int n_total, item_total;
    int pos = block_exclusive_scan(n, warp_tot, &n_total);
    __syncthreads();
    int off = block_exclusive_scan(items, warp_tot, &item_total);
    for (int q = p0; q < p1; ++q) {
        const int p = order[q];
        const BatchProblem& bp = probs[p];
        const int c = bp.list_items[l];
        if (c <= 0 || *bp.ks.all_done) continue;
        L.ids[pos] = p;
        L.prefix[pos] = off;
        ++pos;
        off += c;
    }
    if (threadIdx.x == 0) {
        *L.np = n_total;
        L.prefix[n_total] = item_total;
        totals[l] = item_total;
    }
}

template <int KT, int TC, bool WIDE>
cudaError_t mvm_dp(const BatchProblem* probs, int dp, bool prepass, int parity, DevList L, int blocks,
                   cudaStream_t st) {
    const int pre = prepass ? 1 : 0;
    switch (dp) {
        case 4: batched_mvm_kernel<KT, TC, 4, WIDE><<<blocks, 256, 0, st>>>(probs, L, pre, parity); break;
        case 8: batched_mvm_kernel<KT, TC, 8, WIDE><<<blocks, 256, 0, st>>>(probs, L, pre, parity); break;
        case 12: batched_mvm_kernel<KT, TC, 12, WIDE><<<blocks, 256, 0, st>>>(probs, L, pre, parity); break;
        case 16: batched_mvm_kernel<KT, TC, 16, WIDE><<<blocks, 256, 0, st>>>(probs, L, pre, parity); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <int KT>
cudaError_t mvm_kt(const BatchProblem* probs, int dp, int T, bool prepass, int parity, DevList L, int blocks,
                   cudaStream_t st) {
    if (prepass) return mvm_dp<KT, 1, false>(probs, dp, true, parity, L, blocks, st);
    if (batch_mvm_wide(T)) {
        return batch_mvm_group(T) == 64 ? mvm_dp<KT, 64, true>(probs, dp, false, parity, L, blocks, st)
                                        : mvm_dp<KT, 32, true>(probs, dp, false, parity, L, blocks, st);
    }
    switch (batch_mvm_group(T)) {
        case 1: return mvm_dp<KT, 1, false>(probs, dp, false, parity, L, blocks, st);
        case 2: return mvm_dp<KT, 2, false>(probs, dp, false, parity, L, blocks, st);
        case 4: return mvm_dp<KT, 4, false>(probs, dp, false, parity, L, blocks, st);
        case 8: return mvm_dp<KT, 8, false>(probs, dp, false, parity, L, blocks, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace

bool batch_mvm_wide(int T) { return T >= 17; }
int batch_mvm_group(int T) {
    if (batch_mvm_wide(T)) return T > 32 ? 64 : 32;
    return T <= 1 ? 1 : T <= 2 ? 2 : T <= 4 ? 4 : 8;
}
int64_t batch_mvm_row_tiles(int64_t Npad, int T) { return batch_mvm_wide(T) ? Npad / 64 : Npad / 32; }

cudaError_t launch_batched_setup(const BatchProblem* probs, int phase, uint64_t seed, int Q, DevList L, int blocks,
                                 cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_setup_kernel<<<blocks, 256, 0, st>>>(probs, phase, seed, Q, L);
    return cudaGetLastError();
}

cudaError_t launch_batched_mvm(const BatchProblem* probs, int cls, int T, bool prepass, int parity, DevList L,
                               int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    const int kt = cls / 4, dp = (cls % 4 + 1) * 4;
    return kt == CIQ_RBF ? mvm_kt<CIQ_RBF>(probs, dp, T, prepass, parity, L, blocks, st)
                         : mvm_kt<CIQ_MATERN52>(probs, dp, T, prepass, parity, L, blocks, st);
}

cudaError_t launch_batched_lanczos_step(const BatchProblem* probs, int j, DevList L, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_lanczos_step_kernel<<<blocks, 256, 0, st>>>(probs, j, L);
    return cudaGetLastError();
}

cudaError_t launch_batched_bounds_nodes(const BatchProblem* probs, int Q, double lmax_margin, double lmin_div,
                                        DevList L, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_bounds_nodes_kernel<<<blocks, 32, 0, st>>>(probs, Q, lmax_margin, lmin_div, L);
    return cudaGetLastError();
}

cudaError_t launch_batched_step_scalar(const BatchProblem* probs, int j, bool final_pass, DevList L, int blocks,
                                       cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_step_scalar_kernel<<<blocks, 256, 0, st>>>(probs, j, final_pass ? 1 : 0, L);
    return cudaGetLastError();
}

cudaError_t launch_batched_step_vector(const BatchProblem* probs, int j, DevList L, int blocks, cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_step_vector_kernel<<<blocks, 256, 0, st>>>(probs, j, L);
    return cudaGetLastError();
}

cudaError_t launch_batched_summary(const BatchProblem* probs, int final_j, double* packed, DevList L, int blocks,
                                   cudaStream_t st) {
    if (blocks <= 0) return cudaSuccess;
    batched_summary_kernel<<<blocks, 32, 0, st>>>(probs, final_j, packed, L);
    return cudaGetLastError();
}

cudaError_t launch_rebuild_lists(const BatchProblem* probs, int P, const int* order, const DynLists& lists,
                                 int* totals, cudaStream_t st) {
    rebuild_lists_kernel<<<kBatchDynLists, 1024, 0, st>>>(probs, P, order, lists, totals);
    return cudaGetLastError();
}

}  // namespace ciq
