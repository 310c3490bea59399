// Batched msMINRES-CIQ: one launch per iteration phase over many independent
// problems of uneven size (the per-problem arithmetic is that of krylov.cu and
// mvm_simt.cu; only the mapping of blocks to work differs).
#pragma once

#include "krylov.cuh"
#include "mvm_tc.cuh"

namespace ciq {

// Everything a batched kernel needs about one problem (device array of P).
struct BatchProblem {
    KrylovState<float> ks;
    LanczosState<float> ls;
    MvmArgs<float> mvm[2];      // main-loop MVM by the parity of j
    MvmArgs<float> pre[2];      // pre-pass MVM (one column) by the parity of j
    const float* X;             // caller's points, N x d row-major
    const float* B;             // caller's right-hand sides, T columns of N
    float* out;                 // caller's output, T columns of N
    float* Xp;                  // scaled, padded points (Npad x dp)
    double* nodes;              // NodeSlot block
    double inv_ls;              // 1 / lengthscale
    double noise;               // sigma^2
    double lmin, lmax;          // given bounds (problems without the pre-pass)
    int d;
    int cls;                    // MVM class: kernel type * 4 + dp / 4 - 1
    int mvm_tiles;              // row tiles of the main MVM (items = tiles x groups)
    int mvm_items;
    int pre_tiles;              // row tiles of the pre-pass MVM (= its items)
    TcPoints tcp;               // tensor-core operands (tensor-core batches only)
    int list_items[10];         // work items of this problem in each main-loop list (0: not a member)
};

constexpr int kBatchClasses = 8;            // 2 kernel types x 4 padded dimensions
// Packed per-problem results: summary[8], the NodeSlot block, then the
// largest Ritz value of column 0's msMINRES tridiagonal (0 unless recorded).
constexpr int kSummaryStride = 10 + kNodeCount;   // ..., Ritz maximum, tensor-core timeout flag

// A work list: problems ids[0..*np) with their first work items prefix[k]
// (prefix[*np] = total).  Block b of a batched launch takes the item b: the
// problem is found by binary search over prefix, and blocks past the total
// return at once, so a grid sized from an older (longer) list is safe.
struct DevList {
    int* np;
    int* ids;
    int* prefix;
};

// Problem and local item of block `item`; false past the list's total.
__device__ __forceinline__ bool list_item(const DevList& L, int item, int& p, int& local) {
    const int np = *L.np;
    if (np <= 0 || item >= L.prefix[np]) return false;
    int lo = 0, hi = np - 1;              // largest k with prefix[k] <= item
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (L.prefix[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    p = L.ids[lo];
    local = item - L.prefix[lo];
    return true;
}

// Main-loop lists rebuilt on the device, kBatchDynLists in all.  CUDA-core
// batches: one per MVM class (kernel type x padded dimension), then the
// recurrence lists.  Tensor-core batches: list 0 is the MVM work of every
// problem (both kernel types), list 2 the V split, list 3 the finishing pass
// (one item per row tile and 16 columns).  The last two are the recurrence
// step's vector part (row chunk x column) and scalar part (one per column).
constexpr int kBatchDynLists = kBatchClasses + 2;
constexpr int kListTcSplit = 2;
constexpr int kListTcFinish = 3;
constexpr int kListStepScalar = kBatchClasses + 1;
static_assert(kBatchDynLists == 10, "BatchProblem::list_items size");
struct DynLists {
    DevList l[kBatchDynLists];
};

enum BatchSetupPhase {
    kBatchPrepare = 0,      // scaled points                   items: ceil(Npad dp / 256)
    kBatchReset,            // zero the per-problem counters   items: 1
    kBatchInitRhs,          // copy b, partial ||b||^2         items: chunks x T
    kBatchInitState,        // q_1, state                      items: chunks x T
    kBatchPreInitA,         // Lanczos start vector            items: pre-pass chunks
    kBatchPreInitB,         // normalise it                    items: pre-pass chunks
    kBatchNodesGiven,       // nodes from given bounds         items: 1
    kBatchCombine,          // output                          items: ceil(N / 256) x T
};

// Narrow (one row per lane) or wide (64 x 64 tile) CUDA-core MVM for T
// columns, and its column-group width; the same choice as the single-problem path.
bool batch_mvm_wide(int T);
int batch_mvm_group(int T);
int64_t batch_mvm_row_tiles(int64_t Npad, int T);

cudaError_t launch_batched_setup(const BatchProblem* probs, int phase, uint64_t seed, int Q, DevList L,
                                 int blocks, cudaStream_t st);
cudaError_t launch_batched_mvm(const BatchProblem* probs, int cls, int T, bool prepass, int parity, DevList L,
                               int blocks, cudaStream_t st);
cudaError_t launch_batched_lanczos_step(const BatchProblem* probs, int j, DevList L, int blocks, cudaStream_t st);
cudaError_t launch_batched_bounds_nodes(const BatchProblem* probs, int Q, double lmax_margin, double lmin_div,
                                        DevList L, int blocks, cudaStream_t st);
// The recurrence step in two launches, as for single solves: the scalars of
// every listed column (one item per column; the final decision pass is this
// launch alone), then the vector work (one item per row chunk and column).
cudaError_t launch_batched_step_scalar(const BatchProblem* probs, int j, bool final_pass, DevList L, int blocks,
                                       cudaStream_t st);
cudaError_t launch_batched_step_vector(const BatchProblem* probs, int j, DevList L, int blocks, cudaStream_t st);
// Summary of every listed problem, gathered with its node block into
// packed[p * kSummaryStride ...] (summary[8], then the NodeSlot block).
cudaError_t launch_batched_summary(const BatchProblem* probs, int final_j, double* packed, DevList L, int blocks,
                                   cudaStream_t st);
// Tensor-core batches (mvm_tc.cu): operand preparation (points centre and
// split operands; unit V scales), the per-iteration V split, and the MVM
// over a list of (problem, row tile x split) items.  `pre` selects the
// pre-pass arguments (one column, a 32-column group) instead of the
// main-loop ones.
cudaError_t launch_batched_tc_mean(const BatchProblem* probs, DevList one, int blocks, cudaStream_t st);
cudaError_t launch_batched_tc_points(const BatchProblem* probs, DevList rows256, int blocks, bool half,
                                     cudaStream_t st);
cudaError_t launch_batched_tc_split(const BatchProblem* probs, int parity, DevList L, int blocks, bool half,
                                    bool pre, cudaStream_t st);
// Both kernel types in one launch (the problem selects the body).
cudaError_t launch_batched_tc_mvm(const BatchProblem* probs, int TP, bool half, int parity, bool pre, DevList L,
                                  int blocks, cudaStream_t st);
// Sum the split partials of every row tile and apply the MVM epilogue.
cudaError_t launch_batched_tc_finish(const BatchProblem* probs, int TP, int parity, bool pre, DevList L, int blocks,
                                     cudaStream_t st);
// Set the kernels' shared-memory attributes (before any stream capture).
cudaError_t prepare_batched_tc_mvm(int TP, bool half);

// Rebuild the kBatchDynLists main-loop lists over problems whose columns
// have not all stopped, in the order order[0..P) (a permutation of the
// problems); totals[l] = the new item total of list l.
cudaError_t launch_rebuild_lists(const BatchProblem* probs, int P, const int* order, const DynLists& lists,
                                 int* totals, cudaStream_t st);

}  // namespace ciq
