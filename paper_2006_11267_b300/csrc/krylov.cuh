// Device state and launchers of the msMINRES recurrence and the Lanczos
// bound pre-pass (App. B.2, App. C).
#pragma once

#include "kernels.cuh"

namespace ciq {

// Layout of the small FP64 node block shared by the pre-pass and the solve.
enum NodeSlot {
    kNodeW = 0,                       // w_q, CIQ_MAX_Q entries
    kNodeT = CIQ_MAX_Q,               // t_q, CIQ_MAX_Q entries
    kNodeLmin = 2 * CIQ_MAX_Q,        // lambda_min used
    kNodeLmax,                        // lambda_max used
    kNodeRitzMin,                     // theta_min of the pre-pass
    kNodeRitzMax,                     // theta_max of the pre-pass
    kNodeSumW,                        // sum_q w_q
    kNodeLanczosSteps,                // pre-pass steps actually taken
    kNodeCount
};

// Per-column status codes of a solve.
enum ColStatus {
    kColRunning = 0,
    kColConverged = 1,      // stop rule met
    kColExact = 2,          // Lanczos breakdown: Krylov space invariant, solve exact (or b = 0)
    kColNaN = 3,            // non-finite Lanczos coefficient
    kColMaxIter = 4,        // max_iter reached with tol > 0
    kColFixedIter = 5       // max_iter reached with tol == 0 (fixed-J run)
};

// Output combination.
enum CombineOp {
    kOpInvSqrt = 0,         // a = sum_q w_q x_q
    kOpSqrtIdentity = 1,    // a = (sum_q w_q) b - sum_q w_q t_q x_q
    kOpSqrtMvm = 2          // y = sum_q w_q x_q, a = K y (MVM launched by the caller)
};

// Per-column scalars the split recurrence step publishes (skip flag, alpha
// in two parts, 1/beta_{j+1}, then delta, eps, 1/gamma, c_q tau per shift).
constexpr int kScoStride = 4 + 4 * CIQ_MAX_Q;

template <typename R>
struct KrylovState {
    int64_t N, Npad;
    int T, Q;
    int nparts;                 // MVM row tiles writing partials
    int nchunks;                // row chunks of the recurrence kernel
    int64_t rows_per_chunk;     // multiple of kRowPad
    R* QA;                      // Lanczos vectors, T x Npad each (q_j alternates between QA/QB)
    R* QB;
    R* D;                       // search directions [2][Q][T][Npad]
    R* Y;                       // accumulated sum_q c_q x_q, [T][Npad] (leading part)
    R* Ylo;                     // trailing part of Y (Y + Ylo carries about twice R's precision)
    R* Bw;                      // right-hand sides, [T][Npad]
    double* partials;           // [nparts][T][3] from the MVM epilogue
    double* ynp;                // [2][nchunks][T] partial ||a_j||^2
    double* beta;               // [2][T] beta_j double-buffered by step parity
    double* beta1;              // [T] ||b||
    double* giv;                // [2][Q][T][5] (c_{j-1}, s_{j-1}, c_{j-2}, s_{j-2}, phibar)
    double* phifinal;           // [Q][T] phibar when the column stopped
    int* status;                // [T] ColStatus
    int* iters;                 // [T] steps applied
    int* brk;                   // [T] breakdown / NaN seen at the last step (ColStatus code)
    int* cnt;                   // [jmax + 2] frozen columns seen at step j
    int* all_done;              // 1 once every column is frozen
    const double* nodes;        // NodeSlot block
    double* summary;            // [8] filled by the summary kernel
    double* tri;                // optional: column 0's T_j, diagonal [jmax + 1] then off-diagonal [jmax + 2]
    // Stored-basis form (basis != nullptr): no directions, no Y updates per step.
    R* basis;                   // [jmax + 2][T][Npad]; slot 0 = q_0 = 0, slot j = q_j (slot j + 1 holds p first)
    R* plo = nullptr;           // [T][Npad] or null: trailing part of p (the MVM's float-pair p)
    double* rcoef;              // [jmax][Q][T][4]: 1/gamma_j, delta_j, eps_j, tau_j of shift q at step j
    double* gauss;              // [2][T][4]: LDL^T pivot d_j, u_j^2, sum_k u_k^2/d_k, alpha_1 (parity of j)
    double* bco;                // [jmax + 1][T]: sum_q c_q y_q(j), the coefficient of q_j
    R* sco;                     // [T][kScoStride]: scalars of the split step (single solves)
    double* ycoef;              // optional [jmax + 1][Q][T]: y_q(j) of every shift (backward pass)
    int jmax;
    int op;                     // CombineOp
    int stop_rule;              // ciq_stop_rule
    double tol;
    double breakdown_rtol;
};

template <typename R>
struct LanczosState {
    int64_t N, Npad;
    int nparts, nchunks;
    int64_t rows_per_chunk;
    int iters;                  // J_L
    R* LA;                      // Lanczos vectors (Npad each)
    R* LB;
    double* partials;           // [nparts][3]
    double* ynp;                // [nchunks]
    double* bpar;               // [2] beta_j double-buffered
    double* alpha;              // [iters]
    double* beta;               // [iters + 1]; beta[0] = ||start||
    int* jeff;                  // steps taken (< iters after a breakdown)
    int* done;                  // breakdown flag (skips the remaining launches)
};

template <typename R>
cudaError_t launch_init_rhs(const KrylovState<R>& s, const R* B, cudaStream_t st);
template <typename R>
cudaError_t launch_init_state(const KrylovState<R>& s, cudaStream_t st);
// vector_part = false leaves step 4 to the next MVM (the tensor-core V split
// of the stored-basis form finishes q_{j+1} from the published scalars).
template <typename R>
cudaError_t launch_msminres_step(const KrylovState<R>& s, int j, bool final_pass, cudaStream_t st,
                                 bool vector_part = true);
// Recurrence blocks resident at once on the device (SMs x blocks per SM).
int step_blocks_per_wave();
template <typename R>
cudaError_t launch_combine(const KrylovState<R>& s, R* out, cudaStream_t st);
template <typename R>
cudaError_t launch_summary(const KrylovState<R>& s, int final_j, cudaStream_t st);
// Stored-basis form: back-substitution R_q y_q = tau_q per column and shift,
// then one pass over the basis forming the output (and ||a||^2 partials for
// the summary in the parity slot of final_j).  kOpSqrtMvm leaves the sum in Y.
template <typename R>
cudaError_t launch_basis_combine(const KrylovState<R>& s, R* out, int final_j, cudaStream_t st);

// Backward pass (Eq. ciq_deriv), stored-basis form, FP32 solves over 2T
// columns [B | G] (s.T = 2T; s.ycoef filled by launch_basis_combine).
// Per-shift solutions Xq[q][c][Npad] = V_c y_q for every column, then
// grad[0] = sum_c sum_q c_q y_qc^T (dK/dl) x_qc, grad[1] the same with
// dK/ds = K_XX / s, grad[2] with dK/dsigma^2 = I (device doubles), c_q = -w_q
// (op kOpInvSqrt) or w_q t_q (kOpSqrtIdentity); x_qc from column c, y_qc
// from column T + c.  part: >= vjp_partials(Npad, T, Q) doubles of scratch.
int64_t vjp_partials(int64_t Npad, int T, int Q);
cudaError_t launch_vjp(const KrylovState<float>& s, const float* Xp, int dp, int kt, double lengthscale,
                       double outputscale, float* Xq, double* part, double* grad, cudaStream_t st);

template <typename R>
cudaError_t launch_lanczos_init(const LanczosState<R>& s, const R* start, uint64_t seed,
                                cudaStream_t st);
template <typename R>
cudaError_t launch_lanczos_step(const LanczosState<R>& s, int j, cudaStream_t st);
// theta_min/max of T_J -> bounds (unless fixed) -> nodes, on one device thread.
template <typename R>
cudaError_t launch_bounds_nodes(const LanczosState<R>& s, double* nodes, int Q, double noise,
                                double lmax_margin, double lmin_div, cudaStream_t st);

// Nodes for given bounds on the device (no pre-pass).
cudaError_t launch_nodes_from_bounds(double* nodes, int Q, double lmin, double lmax,
                                     cudaStream_t st);

}  // namespace ciq
