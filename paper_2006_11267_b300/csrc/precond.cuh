// Partial pivoted Cholesky preconditioner of msMINRES-CIQ (App.
// "Preconditioning msMINRES-CIQ"): P = L L^T + sigma^2 I with L the rank-R
// pivoted Cholesky factor of K_XX.
//
// The solve runs msMINRES on the preconditioned operator A = P^{-1/2} K P^{-1/2}
// (whose shifted solves are P^{1/2} (K + t P)^{-1} P^{1/2}) and maps its result
// back with P^{-1/2} (R' b, Eq. precond_sqrt_inverse) or P^{1/2} (R b,
// Eq. precond_sqrt).  The roots of P come in closed form from the
// eigendecomposition L^T L = U diag(s) U^T:
//     Qh = L U diag(s)^{-1/2}      (orthonormal basis of range(L), N x R')
//     P^{+-1/2} = sigma^{+-1} I + Qh diag(g^{+-}) Qh^T,
//     g^- = (s + sigma^2)^{-1/2} - 1/sigma,  g^+ = (s + sigma^2)^{1/2} - sigma.
// Both applications lose at most about sqrt(kappa(P)) digits to cancellation,
// so they run in FP32; P^{-1} alone (the paper's matrix-inversion-lemma form)
// cancels like kappa(P) and does not survive FP32 at sigma^2 = 1e-3.
#pragma once

#include "kernels.cuh"

namespace ciq {

constexpr int kPcMaxRank = 1024;    // largest preconditioner rank
constexpr int kPcMaxTrain = 2048;   // largest rank of a low-rank term (training points of a posterior)

struct PrecondState {
    int64_t N = 0, Npad = 0;
    int rank = 0;                   // R' kept directions (columns of Qh)
    const float* Qh = nullptr;      // [R'][Npad], zero rows past N
    const float* gm = nullptr;      // [R'] g^-
    const float* gp = nullptr;      // [R'] g^+
    float sigma = 0.f, inv_sigma = 0.f;
    float* cpart = nullptr;         // [chunks][T][R'] partial sums of Qh^T X
    float* coef = nullptr;          // [R'][T]
    int T = 0;                      // columns the scratch is sized for
    // Low-rank correction instead of a preconditioner: the MVM is K V + Qh
    // diag(gm) Qh^T V (gm = -1: K - C C^T with C = Qh), no P^{+-1/2}.
    bool lowrank = false;
    const float* mu = nullptr;      // low-rank mode: added to every output column (may be null)
};

int64_t pc_chunks(int64_t Npad);
size_t pc_scratch_floats(int64_t Npad, int rank, int T);

// out = sigma^{e} X + Qh diag(g) Qh^T X with e = -1, g = g^- (inverse root)
// or e = +1, g = g^+ (root).  X: T columns, leading dimension ldx, rows >=
// N read as 0; out: leading dimension ldo, rows >= N written as 0 when
// ldo >= Npad.  stop: skip when *stop != 0 (may be null).
// vscale (optional, with inverse_root and unit columns X): also write the
// tensor-core MVM's power-of-two operand scales of out for TP columns.
cudaError_t launch_pc_apply(const PrecondState& pc, const float* X, int64_t ldx, int T, bool inverse_root,
                            float* out, int64_t ldo, const int* stop, cudaStream_t st, float* vscale = nullptr,
                            int TP = 0);

// Lanczos epilogue of the preconditioned MVM: with O' = K U (U = P^{-1/2} q),
// O = P^{-1/2} O' and p = O - beta q_prev (0 on rows >= N) written to pout
// (over qprev when null); per 128-row tile and column the FP64 sums (q.p,
// p.p, q.q) go to partials[(tile * T + c) * 3 + k].
cudaError_t launch_pc_lanczos(const PrecondState& pc, const float* Oraw, const float* q, float* qprev, float* pout,
                              const double* beta, double* partials, int T, const int* stop, cudaStream_t st);

// Rows of 128 of the epilogue's partial sums.
inline int64_t pc_row_tiles(int64_t Npad) { return Npad / 128; }

// ---- setup ----
// Pivoted Cholesky of K_XX from the scaled points (Npad x dp, divided by the
// lengthscale): L [rank][Npad] (column m contiguous), piv [rank] pivots,
// dres [Npad] (FP64 scratch, left holding the residual diagonal), and
// `work` of pc_cholesky_work_bytes(Npad) bytes.  *rank_out (device int) is
// the number of columns formed (smaller when the residual diagonal vanishes).
size_t pc_cholesky_work_bytes(int64_t Npad);
// With Ct (device, [rk][Npad], rk <= kPcMaxTrain), the factor is that of
// K_XX - C C^T (its columns and diagonal lose the low-rank term).
cudaError_t launch_pivoted_cholesky(const float* Xp, int64_t N, int64_t Npad, int dp, int kt, float outputscale,
                                    int rank, float* L, int* piv, double* dres, void* work, int* rank_out,
                                    cudaStream_t st, const float* Ct = nullptr, int rk = 0);

// G = L^T L (FP64, R x R, column-major) from L [R][Npad]; gpart: scratch of
// pc_gram_scratch(Npad, R) doubles.
int64_t pc_gram_scratch(int64_t Npad, int R);
cudaError_t launch_gram(const float* L, int64_t Npad, int R, double* gpart, double* G, cudaStream_t st);

// Qh[c][i] = sum_m L[m][i] W[m][c] (FP64 accumulation, rounded once):
// W is R x Rk column-major FP64 (device).
cudaError_t launch_basis_from_factor(const float* L, int64_t Npad, int R, const double* W, int Rk, float* Qh,
                                     cudaStream_t st);

// out[c][i] = sum_m A[m][i] W[m][c] with FP64 A [R][Npad] (FP64 accumulation,
// rounded once to FP32).
cudaError_t launch_product_f64(const double* A, int64_t Npad, int R, const double* W, int Rk, float* out,
                               cudaStream_t st);

// Lanczos epilogue of an MVM with a low-rank correction, O = O' + Qh diag(gm)
// Qh^T V (V: the MVM's input, O': its plain output, both leading dimension
// Npad), then p = O - beta q_prev and the partial sums as launch_pc_lanczos.
// With gm = -1 this is (K - C C^T) V for C = Qh.
// O += Qh diag(gm) Qh^T V in place (O, V: leading dimension Npad): the
// low-rank term of the MVM on its own (gm = -1: O - C C^T V).
cudaError_t launch_lowrank_apply(const PrecondState& lr, const float* V, float* O, int T, const int* stop,
                                 cudaStream_t st);

cudaError_t launch_lowrank_lanczos(const PrecondState& pc, const float* V, const float* Oraw, const float* q,
                                   float* qprev, float* pout, const double* beta, double* partials, int T,
                                   const int* stop, cudaStream_t st);

}  // namespace ciq
