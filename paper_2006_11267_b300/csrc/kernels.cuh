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
    R* pout;               // kLanczos: where p goes (nullptr: over q_prev)
    // Optional (tensor-core MVM only): V holds p of the previous step and the
    // V split first finishes that step's Lanczos update in place, V = (V -
    // alpha q) / beta per column from lz_sco rows [skip, alpha_hi, alpha_lo,
    // 1/beta] (kScoStride apart; skip != 0 leaves the column as it is).
    const R* lz_q;
    const R* lz_sco;
    const double* beta;    // kLanczos: beta_j per column
    double* partials;      // kLanczos: [ntiles][T][3]
    const int* stop;       // optional: skip the launch when *stop != 0
    // Optional (CUDA-core MVM, kLanczos): p as a float pair.  p is formed in
    // FP64 from the MVM's compensated sum, its leading part goes where p
    // goes and its trailing part to plo (T x ldv), and the partial sums use
    // the unrounded p.
    R* plo = nullptr;
};

// Epilogue of one output entry O[i][col] (before the noise term): kPlain
// stores O + sigma^2 v; kLanczos forms p = O + sigma^2 v - beta q_prev (0 on
// padded rows), writes it to pout (over q_prev when pout is null) and
// accumulates q.p, p.p, q.q in FP64.
// PAIR: the caller supplies the trailing part olo of its sum and honours
// a.plo (the CUDA-core MVMs); without it the float-pair branch is not
// compiled in (it would change the register allocation of the stored-K
// kernels' main loops: measured 2x slower at T = 8).
template <typename R, bool PAIR = false>
__device__ __forceinline__ void lanczos_epilogue_value(const MvmArgs<R>& a, int64_t i, int col, R o,
                                                       double& qp, double& pp, double& qq, R olo = (R)0) {
    const int64_t idx = (int64_t)col * a.ldv + i;
    const R v = a.V[idx];
    if (PAIR && a.mode == kLanczos && a.plo) {
        // o + olo is the MVM's sum as a pair; p = O + sigma^2 v - beta q_prev in FP64.
        const double pd = i < a.N ? (double)o + (double)olo + (double)a.noise * (double)v -
                                        a.beta[col] * (double)a.qprev[idx]
                                  : 0.0;
        const R ph = (R)pd;
        (a.pout ? a.pout : a.qprev)[idx] = ph;
        a.plo[idx] = (R)(pd - (double)ph);
        qp += (double)v * pd;
        pp += pd * pd;
        qq += (double)v * (double)v;
        return;
    }
    o += a.noise * v;
    if (a.mode == kPlain) {
        if (i < a.N) a.out[(int64_t)col * a.ldo + i] = o;
        return;
    }
    R p = (i < a.N) ? (R)(o - (R)a.beta[col] * a.qprev[idx]) : (R)0;
    (a.pout ? a.pout : a.qprev)[idx] = p;
    qp += (double)v * (double)p;
    pp += (double)p * (double)p;
    qq += (double)v * (double)v;
}

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
