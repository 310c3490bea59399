// Internal launch interfaces of libciq.
#pragma once

#include "common.cuh"

namespace ciq {

// Epilogue of a kernel MVM O = (K_XX + sigma^2 I) V over one row tile.
//  kPlain:   out[c*ldo + i] = O[i][c]
//  kLanczos: p = O[i][c] - beta[c] * qprev[c*ldv + i] is written over qprev
//            (rows >= N get 0), and per row tile and column the FP64 sums
//            (q.p, p.p, q.q) with q = V go to partials[(tile*T + c)*3 + k].
enum MvmMode { kPlain = 0, kLanczos = 1 };

template <typename R>
struct MvmArgs {
    const R* X;            // Npad x dp, points divided by the lengthscale, zero rows past N
    int64_t N;
    int64_t Npad;          // multiple of kRowPad
    int dp;                // padded dimension (multiple of 4, <= kMaxDimPad)
    int kt;                // ciq_kernel_type
    R s;                   // outputscale
    R noise;               // sigma^2
    const R* V;            // T columns, leading dimension ldv (= Npad)
    int64_t ldv;
    int T;
    int mode;              // MvmMode
    R* out;                // kPlain
    int64_t ldo;
    R* qprev;              // kLanczos
    const double* beta;    // kLanczos: beta_j per column
    double* partials;      // kLanczos: [ntiles][T][3]
    const int* stop;       // optional: skip the launch when *stop != 0
};

// Number of row tiles (entries of `partials`) the SIMT MVM uses for T columns.
template <typename R>
int64_t mvm_simt_row_tiles(int64_t Npad, int T);

template <typename R>
cudaError_t launch_mvm_simt(const MvmArgs<R>& a, cudaStream_t st);

// Points scaled by 1/lengthscale into Xp (Npad x dp, zero padded).
template <typename R, typename Rin>
cudaError_t launch_prepare_points(const Rin* X, int64_t N, int d, int64_t Npad, int dp,
                                  double inv_ls, R* Xp, cudaStream_t st);

}  // namespace ciq
