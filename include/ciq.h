/*
 * ciq.h -- C ABI of libciq: msMINRES-CIQ square roots of Gaussian-process
 * kernel matrices on one B300 (sm_103a).
 *
 * Method: Pleiss, Jankowiak, Eriksson, Damle, Gardner, "Fast Matrix Square
 * Roots with Applications to Gaussian Processes and Bayesian Optimization"
 * (NeurIPS 2020).  For K = K_XX + sigma^2 I the library returns
 *
 *     K^{-1/2} B ~= sum_q w_q (t_q I + K)^{-1} B          (Eq. contour_integral_quad)
 *     K^{1/2}  B ~= K sum_q w_q (t_q I + K)^{-1} B
 *
 * with nodes (w_q, t_q) from Jacobi elliptic functions over Lanczos-estimated
 * spectral bounds (App. B, Algorithm "quadrature") and the Q shifted solves
 * done together by one multi-shift MINRES (App. C, Algorithm "msMINRES"),
 * one kernel MVM per iteration regardless of Q (Property 1).
 *
 * Kernels (the paper names them but does not write them out; this is the
 * convention of the library, r = ||x - x'||, l = lengthscale, s = outputscale):
 *     CIQ_RBF       k(r) = s exp(-r^2 / (2 l^2))
 *     CIQ_MATERN52  k(r) = s (1 + sqrt5 r/l + 5 r^2/(3 l^2)) exp(-sqrt5 r/l)
 *
 * Layout (all calls):
 *   X    row-major N x d single (or double for *_f64) precision: point i is
 *        X[i*d .. i*d + d-1].  1 <= d <= CIQ_MAX_DIM.
 *   B    T right-hand sides of N entries each, back to back: entry i of
 *        column c is B[c*N + i] (column-major N x T, leading dimension N).
 *   out  same layout as B.
 *
 * Memory: X, B, out, the Lanczos start vector and the optional nodes may be
 * host or device pointers (checked with cudaPointerGetAttributes).  Host
 * buffers are copied to and from the device inside the call.  The caller
 * owns every buffer it passes.  The library owns its workspace unless
 * ciq_options.workspace is set.
 *
 * Errors: no call aborts, traps or prints.  Every call returns a ciq_status.
 * CIQ_NOT_CONVERGED still writes the final iterate and fills the info.
 *
 * Streams: work is queued on `stream` (NULL = legacy default stream).  The
 * solve entry points return after the result is written (they read a device
 * convergence flag between batches of iterations), so they are synchronous
 * with respect to `stream`.
 */
#ifndef CIQ_H
#define CIQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st* ciq_stream_t;

#define CIQ_MAX_DIM 16        /* largest point dimension d */
#define CIQ_MAX_Q 32          /* largest number of quadrature points Q */
#define CIQ_MAX_BATCH 65536   /* largest number of problems of one batched call */
#define CIQ_MAX_TRAIN 2048    /* largest training set of ciq_posterior_sample */

typedef enum {
    CIQ_OK = 0,
    CIQ_ERR_ARG = 1,          /* bad size, NULL pointer, bad enum, Q/d out of range */
    CIQ_ERR_CUDA = 2,         /* a CUDA runtime call failed (no device, launch error) */
    CIQ_ERR_NOMEM = 3,        /* device workspace could not be allocated */
    CIQ_NOT_CONVERGED = 4,    /* max_iter reached before every column met the stop rule */
    CIQ_ERR_NAN = 5,          /* a non-finite Lanczos coefficient appeared */
    CIQ_ERR_UNSUPPORTED = 6,  /* valid request this build does not implement */
    CIQ_ERR_SCRATCH_TOO_SMALL = 7, /* problem larger than the static scratch of ciq_kernel_mvm_noalloc */
    CIQ_ERR_TIMEOUT = 8       /* a bounded wait of the tensor-core MVM gave up (about 2 s); the
                                 kernel stopped cleanly, later MVMs of the call were skipped and the
                                 results are invalid; the device stays usable.  Reported by the
                                 solves (which wait for their stream); ciq_kernel_mvm returns
                                 before its kernels finish and does not report it */
} ciq_status;

typedef enum { CIQ_RBF = 0, CIQ_MATERN52 = 1 } ciq_kernel_type;

/* Kernel hyperparameters; noise is sigma^2 added to the diagonal of K_XX. */
typedef struct {
    int type;                 /* ciq_kernel_type */
    double lengthscale;       /* > 0 */
    double outputscale;       /* > 0 */
    double noise;             /* >= 0 */
} ciq_kernel;

/* Arithmetic of the kernel tiles inside the MVM (vectors stay FP32,
 * Lanczos/Givens scalars stay FP64 in every mode). */
typedef enum {
    CIQ_PREC_FP32 = 0,        /* plain FP32 on CUDA cores */
    CIQ_PREC_TF32 = 1,        /* tensor cores (tcgen05, kind::tf32): P and V rounded to TF32, one
                                 product, no split (the distance tile keeps the FP16 split);
                                 single problems only (batches: CIQ_ERR_UNSUPPORTED) */
    CIQ_PREC_BF16 = 2,        /* tensor cores (tcgen05): every operand split into two BF16 parts */
    CIQ_PREC_FP16 = 3         /* tensor cores (tcgen05): every operand split into two FP16 parts */
} ciq_precision;

typedef enum {
    CIQ_MVM_AUTO = 0,         /* on-the-fly */
    CIQ_MVM_ONTHEFLY = 1,     /* K recomputed tile by tile every MVM, never stored */
    CIQ_MVM_STORED = 2        /* K formed once in the workspace (Npad^2 floats, FP32), streamed
                                 every iteration; FP32 precision only */
} ciq_mvm_mode;

typedef enum {
    CIQ_STOP_RESIDUAL = 0,    /* per column: max_q |phibar_q| / ||b|| <= tol */
    CIQ_STOP_ERRBOUND = 1     /* per column: sum_q c_q |phibar_q| / (t_q + lmin) <= tol ||a_j|| */
} ciq_stop_rule;

/* How the iterates are formed (single solves; batched solves always recur).
 * RECURRENCE is App. C as written: Q search directions per column, updated every
 * step, O(QNT) memory.  BASIS keeps every Lanczos vector in the workspace
 * ((max_iter + 2) T Npad floats) and forms the Q solutions once at the end,
 * x_q = V_J R_q^{-1} tau_q, from the FP64 Givens factors recorded every step:
 * the same MINRES iterates with (3Q + 4) fewer vector passes per iteration.
 * Under CIQ_STOP_ERRBOUND, BASIS compares the bound with tol (1 - 2 tol)
 * times ||K^{1/2}b|| = ||b|| sqrt(alpha_1) (square root; the CIQ_SQRT_MVM
 * form's bound is multiplied by lmax_used) or times the Gauss-quadrature lower
 * bound of ||K^{-1/2}b|| from T_j (inverse root), instead of tol times the
 * running estimate's norm; the bound is then <= tol ||a_j|| as well.  AUTO: BASIS for FP32 solves whose basis takes at
 * most a quarter of the device memory, else RECURRENCE.  In either form an FP32
 * solve whose MVM runs on CUDA cores (batched problems included) forms the Lanczos
 * p = O + sigma^2 v - beta q_{j-1} in FP64 from the MVM's compensated sum and keeps
 * it as a float pair (T Npad more floats of workspace); q_{j+1} is rounded once. */
typedef enum {
    CIQ_KRYLOV_AUTO = 0,
    CIQ_KRYLOV_RECURRENCE = 1,
    CIQ_KRYLOV_BASIS = 2
} ciq_krylov_form;

typedef enum {
    CIQ_SQRT_IDENTITY = 0,    /* K^{1/2}b = (sum w_q) b - sum w_q t_q x_q   (no extra MVM) */
    CIQ_SQRT_MVM = 1          /* K^{1/2}b = K (sum w_q x_q)                 (one extra MVM) */
} ciq_sqrt_form;

typedef struct {
    int precision;            /* ciq_precision (default CIQ_PREC_FP32) */
    int mvm;                  /* ciq_mvm_mode (default CIQ_MVM_AUTO) */
    int stop_rule;            /* ciq_stop_rule (default CIQ_STOP_RESIDUAL) */
    int sqrt_form;            /* ciq_sqrt_form (default CIQ_SQRT_IDENTITY) */
    int max_iter;             /* J_max, msMINRES iterations (default 200) */
    int lanczos_iters;        /* J_L, Lanczos steps of the bound pre-pass (default 10) */
    int check_every;          /* iterations queued between convergence reads (default 8) */
    int profile;              /* 1: time every kernel launch with CUDA events (fills info->t_*) */
    uint64_t seed;            /* start vector seed when lanczos_start is NULL */
    const float* lanczos_start; /* optional N entries (host or device; FP64 calls read double*) */
    double lmax_margin;       /* lambda_max_used = lmax_margin * theta_max (default 1.05) */
    double lmin_div;          /* lambda_min_used = theta_min / lmin_div if noise == 0 (default 100) */
    double lmin, lmax;        /* both > 0: use these bounds and skip the pre-pass */
    const double* quad_w;     /* optional Q weights (host); with quad_t skips pre-pass and nodes */
    const double* quad_t;     /* optional Q shifts (host) */
    void* workspace;          /* optional device workspace of workspace_bytes */
    size_t workspace_bytes;
    int graph;                /* batched solves: capture each batch of check_every iterations as a
                                 CUDA graph and launch it as one (default 1); single solves ignore it */
    int tc_split;             /* tensor-core MVM: CTAs sharing one 128-row tile (1..8; 0 = chosen
                                 from N for single solves, 1 for batched solves) */
    int fault_inject;         /* testing only (default 0): 1 makes CTA 0 of the first tensor-core MVM
                                 skip its first point copy, so its bounded waits run out and the
                                 call returns CIQ_ERR_TIMEOUT (the failure-detection path) */
    int krylov;               /* ciq_krylov_form (default CIQ_KRYLOV_AUTO) */
    int batch_split_rows;     /* tensor-core batches: problems of at least this many 128-row tiles
                                 run batch_split CTAs per row tile (0 = off, the default) */
    int batch_split;          /* 1..8 (used when batch_split_rows > 0) */
    int precond_rank;         /* ciq_posterior_sample: rank of a pivoted-Cholesky preconditioner of
                                 COV* (0 = none, the default; 1..1024); the draws then use the
                                 rotated root R (R R^T = COV*) instead of the principal one */
} ciq_options;

typedef struct {
    int iters;                /* msMINRES iterations of the slowest column (= MVMs) */
    int iters_min;            /* ... of the fastest column */
    int converged;            /* columns that met the stop rule */
    int lanczos_iters;        /* MVMs spent in the bound pre-pass */
    double resid_max;         /* max over columns, shifts of |phibar_q| / ||b|| */
    double errbound_max;      /* max over columns of sum_q c_q|phibar_q|/(t_q+lmin) / ||a|| */
    double ritz_min, ritz_max;/* extreme Ritz values of the pre-pass (0 if skipped) */
    double lmin_used, lmax_used;
    double w[CIQ_MAX_Q];      /* nodes used */
    double t[CIQ_MAX_Q];
    int q;
    int launches;             /* kernels launched by the call */
    double t_total_ms;        /* profile: device time of the whole call */
    double t_prepass_ms;      /* profile: Lanczos pre-pass and nodes */
    double t_mvm_ms;          /* profile: sum over msMINRES kernel-MVM launches */
    double t_step_ms;         /* profile: sum over msMINRES recurrence launches */
    int mvm_launches;         /* profile: msMINRES kernel-MVM launches timed */
    int step_launches;        /* profile: recurrence launches timed */
    double ritz_max_solve;    /* largest Ritz value of column 0's msMINRES tridiagonal
                                 (ciq_*_batched_learned only; else 0) */
    int krylov;               /* ciq_krylov_form the solve ran (RECURRENCE or BASIS) */
    int precond_rank;         /* ciq_*_precond: directions of the preconditioner kept (else 0) */
} ciq_info;

/* Human-readable name of a status code (static string). */
const char* ciq_status_string(int status);

/* Fill *opt with the defaults listed in ciq_options. */
void ciq_default_options(ciq_options* opt);

/* Quadrature weights and shifts for K^{-1/2} ~= sum_q w_q (t_q I + K)^{-1}.
 * Eq. quad_points_and_locations with the sign flip of Eq.
 * contour_integral_quad_4 and Algorithm "quadrature" (App. B), FP64 on the
 * host: k^2 = lmin/lmax, K' = K(k'), u_q = (q - 1/2)/Q, Jacobi elliptic
 * functions at u_q K' with parameter 1 - k^2, Jacobi imaginary transform.
 * w, t: host arrays of Q doubles written by the call.  Requires
 * 0 < lmin <= lmax and 1 <= Q <= CIQ_MAX_Q, else CIQ_ERR_ARG. */
ciq_status ciq_quad_nodes(double lmin, double lmax, int Q, double* w, double* t);

/* Extreme Ritz values of `iters` Lanczos steps on K = K_XX + sigma^2 I from
 * a random start (App. B.2; Algorithm "quadrature", first two lines), and the
 * bounds the solves use: lmax_used = 1.05 theta_max; lmin_used = sigma^2 when
 * sigma^2 > 0 (K_XX is PSD), else theta_min / 100.  All outputs are host
 * doubles; any may be NULL.  `start` (N floats, host or device) may be NULL:
 * the start vector is then 2u - 1 with u the splitmix64 uniforms of `seed`.
 * 1 <= iters <= 512. */
ciq_status ciq_lanczos_bounds(const float* X, int64_t N, int d, const ciq_kernel* kern,
                              int iters, uint64_t seed, const float* start,
                              double* ritz_min, double* ritz_max,
                              double* lmin_used, double* lmax_used, ciq_stream_t stream);

/* K^{1/2} B (Eq. contour_integral_quad, right) and K^{-1/2} B (left) by
 * msMINRES-CIQ (Algorithm "ciq").  Q in [1, CIQ_MAX_Q]; tol >= 0 (0 runs
 * max_iter iterations); T >= 1; N >= 1.  `opt` may be NULL (defaults);
 * `info` may be NULL.  FP32 vectors, FP64 Lanczos/Givens scalars. */
ciq_status ciq_sqrt(const float* X, int64_t N, int d, const ciq_kernel* kern,
                    const float* B, int T, int Q, double tol, const ciq_options* opt,
                    float* out, ciq_info* info, ciq_stream_t stream);
ciq_status ciq_invsqrt(const float* X, int64_t N, int d, const ciq_kernel* kern,
                       const float* B, int T, int Q, double tol, const ciq_options* opt,
                       float* out, ciq_info* info, ciq_stream_t stream);

/* Same in FP64 end to end (kernel tiles, vectors and scalars).  opt->precision
 * and opt->mvm are ignored (FP64 on-the-fly); lanczos_start, if set, points
 * to N doubles. */
ciq_status ciq_sqrt_f64(const double* X, int64_t N, int d, const ciq_kernel* kern,
                        const double* B, int T, int Q, double tol, const ciq_options* opt,
                        double* out, ciq_info* info, ciq_stream_t stream);
ciq_status ciq_invsqrt_f64(const double* X, int64_t N, int d, const ciq_kernel* kern,
                           const double* B, int T, int Q, double tol, const ciq_options* opt,
                           double* out, ciq_info* info, ciq_stream_t stream);

/* out = (K_XX + sigma^2 I) V, the MVM of every msMINRES iteration (Property 1,
 * Sec. 3.3), with K never stored (on-the-fly tiles).  V, out: device, T
 * columns of N floats.  precision: ciq_precision.  Asynchronous on stream. */
ciq_status ciq_kernel_mvm(const float* X, int64_t N, int d, const ciq_kernel* kern,
                          const float* V, int T, float* out, int precision,
                          ciq_stream_t stream);
ciq_status ciq_kernel_mvm_f64(const double* X, int64_t N, int d, const ciq_kernel* kern,
                              const double* V, int T, double* out, ciq_stream_t stream);

/* Stored K for the stored-K MVM (the explicit-matrix case of Sec. 3.3,
 * O(J N^2) with K resident): K = K_XX + sigma^2 I written in FP32 into
 * device memory Kmat laid out as Npad = round_up(N, 128) rows of ldk floats
 * (ldk >= Npad, ldk % 4 == 0); rows and columns in [N, Npad) are set to 0.
 * The caller allocates Npad * ldk floats.  X: device.  Asynchronous on
 * stream; CIQ_ERR_ARG on a bad size or host pointer. */
ciq_status ciq_kernel_matrix(const float* X, int64_t N, int d, const ciq_kernel* kern,
                             float* Kmat, int64_t ldk, ciq_stream_t stream);

/* out = Kmat V for a matrix in the layout ciq_kernel_matrix writes (Npad
 * rows of ldk floats, zero padding).  V, out: device, T columns of N floats.
 * precision CIQ_PREC_FP32: CUDA cores, compensated accumulation, HBM-bound
 * for T <= 16.  CIQ_PREC_FP16 / BF16: tensor cores; K (read once by TMA,
 * Kmat 16-byte aligned) is scaled by a power of two taken from its largest
 * diagonal entry (which bounds every entry of a positive semidefinite K;
 * entries beyond 2^15 times it overflow) and split into two 16-bit parts, V
 * likewise (about 22 significant bits with FP16 parts); this call reads the
 * diagonal maximum back to the host (it synchronises the stream once).
 * CIQ_PREC_TF32: CIQ_ERR_UNSUPPORTED.  Asynchronous on stream otherwise. */
ciq_status ciq_stored_mvm(const float* Kmat, int64_t N, int64_t ldk, const float* V, int T,
                          float* out, int precision, ciq_stream_t stream);

/* K^{1/2} B and K^{-1/2} B for a caller's explicit symmetric positive
 * definite K: the general-matrix case of Sec. 3.3 (any K with an MVM; here
 * the stored-K MVM, O(J N^2) per solve), used e.g. for matrices with a
 * prescribed spectrum (Sec. 5, Fig. quad_error).  K: N x N row-major floats
 * with leading dimension ldk >= N, host or device (copied once into the
 * workspace's zero-padded Npad x Npad layout; only the FP32 path exists, so
 * opt->precision must be CIQ_PREC_FP32, else CIQ_ERR_UNSUPPORTED).  B, out,
 * opt, info and the return codes are those of ciq_sqrt.  There is no noise
 * term: without opt->lmin/lmax the pre-pass bounds are lambda_max =
 * lmax_margin theta_max and lambda_min = theta_min / lmin_div (reading R4 for
 * sigma^2 = 0).  Workspace: ciq_workspace_bytes(N, 1, T, Q, opt with mvm =
 * CIQ_MVM_STORED). */
ciq_status ciq_sqrt_dense(const float* K, int64_t N, int64_t ldk, const float* B, int T, int Q, double tol,
                          const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream);
ciq_status ciq_invsqrt_dense(const float* K, int64_t N, int64_t ldk, const float* B, int T, int Q, double tol,
                             const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream);

/* Backward pass (Sec. 3.4, Eq. ciq_deriv): the forward result out = K^{-1/2}B
 * (ciq_invsqrt_vjp) or K^{1/2}B (ciq_sqrt_vjp, identity form), and for the loss
 * L = sum_c G_c . out_c its gradients grad_B = dL/dB (T x N like B) and
 * grad_theta[0..2] = dL/d lengthscale, dL/d outputscale, dL/d noise (host, summed
 * over the T columns).  The quadrature is differentiated term by term with its
 * nodes held fixed: dL/dtheta = sum_q c_q y_q^T (dK/dtheta) x_q with x_q, y_q the
 * shifted solves of b and g (c_q = -w_q, or w_q t_q for the square root), and
 * dL/dB is the same root applied to G.  One solve runs over the 2T columns
 * [B | G] in the stored-basis form (opt->krylov RECURRENCE or opt->sqrt_form
 * CIQ_SQRT_MVM: CIQ_ERR_UNSUPPORTED); the contractions then run on CUDA cores
 * over all N^2 kernel entries (O(N^2 Q T) work).  X, B, G, out, grad_B: host or
 * device; precision, stop rule and bounds as in ciq_sqrt, applied to all 2T
 * columns.  Returns after the stream work. */
ciq_status ciq_invsqrt_vjp(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, const float* G,
                           int T, int Q, double tol, const ciq_options* opt, float* out, float* grad_B,
                           double* grad_theta, ciq_info* info, ciq_stream_t stream);
ciq_status ciq_sqrt_vjp(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, const float* G,
                        int T, int Q, double tol, const ciq_options* opt, float* out, float* grad_B,
                        double* grad_theta, ciq_info* info, ciq_stream_t stream);

/* One problem of a batch: X (device, N x d), B and out (device, T columns of
 * N floats).  lmin, lmax > 0 give this problem's spectral bounds and skip its
 * Lanczos pre-pass (e.g. bounds predicted by a learned model); otherwise the
 * pre-pass runs as in ciq_sqrt. */
typedef struct {
    const float* X;
    int64_t N;
    int d;
    ciq_kernel kern;
    const float* B;
    int T;
    float* out;
    double lmin, lmax;
} ciq_problem;

/* K_p^{1/2} B_p / K_p^{-1/2} B_p for P independent problems of uneven N and d
 * (the batched form of Algorithm "ciq"): one launch per iteration phase
 * covers every problem that has not stopped (work lists rebuilt on the device
 * between batches of iterations, finished problems drop out); problems share
 * Q, tol and the options; all problems must have the same T.  FP32 vectors,
 * FP64 scalars; on-the-fly MVM on CUDA cores (CIQ_PREC_FP32) or on tensor
 * cores with FP16/BF16 split tiles (CIQ_PREC_FP16/BF16; then T <= 64 and
 * every d <= 14; CIQ_PREC_TF32: CIQ_ERR_UNSUPPORTED).  Every problem's arithmetic is that of ciq_sqrt /
 * ciq_invsqrt with the same options, so each output equals the
 * single-problem call's bit for bit (tensor-core batches run one CTA per
 * row tile unless opt->tc_split says otherwise, so the single call is
 * compared with the same tc_split).  The work lists hold the problems in
 * decreasing padded N (longest CTAs first); order and batch composition
 * change only the schedule, never a result.  1 <= P <= CIQ_MAX_BATCH.
 * CIQ_ERR_UNSUPPORTED if opt->mvm is CIQ_MVM_STORED, opt->sqrt_form is not
 * CIQ_SQRT_IDENTITY, quad_w, quad_t, lanczos_start or workspace is set, or a
 * tensor-core batch breaks its limits.  The device workspace (the sum of
 * the problems' ciq_workspace_bytes plus small tables) is allocated on
 * stream and freed before return; the call returns after the stream work.
 * infos: NULL or P entries (launches = the call's total).  Returns
 * CIQ_ERR_NAN / CIQ_NOT_CONVERGED if any problem ended so, CIQ_ERR_ARG on a
 * bad problem or a host pointer (nothing is computed). */
ciq_status ciq_sqrt_batched(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                            ciq_info* infos, ciq_stream_t stream);
ciq_status ciq_invsqrt_batched(const ciq_problem* probs, int P, int Q, double tol,
                               const ciq_options* opt, ciq_info* infos, ciq_stream_t stream);

/* ---- learned spectral-bound predictor (no counterpart in the paper) ----
 *
 * A regression network (CIQ_MLP_INPUTS -> 64 tanh -> 64 tanh ->
 * CIQ_MLP_OUTPUTS) that predicts, from a problem's description, what the
 * Lanczos pre-pass and the msMINRES run would report: log theta_min,
 * log theta_max (the pre-pass's Ritz extremes, App. B.2) and log of the
 * iteration count.  Used by ciq_*_batched_learned to skip the pre-pass.
 *
 * Inputs of a problem (float[CIQ_MLP_INPUTS]): log N, d, kernel type (0 RBF,
 * 1 Matern-5/2), log lengthscale, log outputscale, log max(sigma^2, 1e-12),
 * the mean of each of the CIQ_MAX_DIM coordinates of X, then the population
 * variance of each (0 for coordinates >= d).
 *
 * Parameters (float[CIQ_MLP_PARAMS], device): input means [0,38), input
 * standard deviations [38,76), output means [76,79), output standard
 * deviations [79,82), then W1 (38 x 64, input-major), b1[64], W2 (64 x 64),
 * b2[64], W3 (64 x 3), b3[3].  Loss: mean over samples and outputs of the
 * squared error of the standardised outputs.  All arrays below are device
 * pointers, row-major (one sample per row); calls are asynchronous on
 * stream unless stated. */
#define CIQ_MLP_INPUTS 38
#define CIQ_MLP_OUTPUTS 3
#define CIQ_MLP_PARAMS 6933

/* F[p * CIQ_MLP_INPUTS ..] = inputs of problem p (X read from the device). */
ciq_status ciq_mlp_features(const ciq_problem* probs, int P, float* F, ciq_stream_t stream);
/* theta[0, 82) = column means and standard deviations of F (n x 38) and
 * Y (n x 3); a constant column gets standard deviation 1. */
ciq_status ciq_mlp_normaliser(const float* F, const float* Y, int n, float* theta, ciq_stream_t stream);
/* Glorot-uniform weights, zero biases: entry k of a weight matrix with fan
 * in a and fan out b is sqrt(6/(a+b)) (2u_k - 1), u_k the splitmix64 uniform
 * number k of seed.  theta[0, 82) is left as it is. */
ciq_status ciq_mlp_init(float* theta, uint64_t seed, ciq_stream_t stream);
/* Full-batch loss (host double) and its gradient grad[CIQ_MLP_PARAMS]
 * (device doubles, 0 on the normaliser entries), FP32 arithmetic. */
ciq_status ciq_mlp_loss_grad(const float* theta, const float* F, const float* Y, int n, double* loss,
                             double* grad, ciq_stream_t stream);
/* Adam steps first_step .. first_step + steps - 1 (bias-corrected; moments
 * 0.9, 0.999, eps 1e-8) on minibatches of `batch` rows drawn with
 * replacement: row k of step t is floor(u n), u the splitmix64 uniform number
 * (t-1) batch + k of seed.  adam: 2 x CIQ_MLP_PARAMS floats (first, second
 * moments), zero before the first step.  losses: NULL or `steps` floats
 * (the minibatch loss before each step).  One CTA runs all steps. */
ciq_status ciq_mlp_train(float* theta, float* adam, const float* F, const float* Y, int n, int steps, int batch,
                         float lr, uint64_t seed, int first_step, float* losses, ciq_stream_t stream);
/* out (n x 3) = predictions in the output units; bf16 != 0 rounds the
 * weights and the activations between layers to BF16 (FP32 accumulation). */
ciq_status ciq_mlp_predict(const float* theta, const float* F, int n, float* out, int bf16, ciq_stream_t stream);

/* The batched solves with bounds from the network instead of the pre-pass.
 * For problem p with predictions (l0, l1, l2): lmax = opt->lmax_margin
 * exp(l1 + margin), lmin = sigma^2 if sigma^2 > 0, else exp(l0) /
 * opt->lmin_div (BF16 inference).  Problems whose own lmin, lmax are set keep
 * them.  After the solve, the largest Ritz value of each problem's msMINRES
 * tridiagonal (column 0, all its iterations) is checked against the lmax
 * used: a problem whose Krylov space shows an eigenvalue above it, or whose
 * solve produced a non-finite coefficient, is solved again with the Lanczos
 * pre-pass (fallback[p] = 1, host int array, may be NULL).  infos as in
 * ciq_sqrt_batched (of the solve whose output is kept); theta: device. */
ciq_status ciq_sqrt_batched_learned(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                                    const float* theta, double margin, ciq_info* infos, int* fallback,
                                    ciq_stream_t stream);
ciq_status ciq_invsqrt_batched_learned(const ciq_problem* probs, int P, int Q, double tol,
                                       const ciq_options* opt, const float* theta, double margin,
                                       ciq_info* infos, int* fallback, ciq_stream_t stream);

/* ---- preconditioned solves (Sec. 3 "Preconditioning"; App. "Preconditioning
 * msMINRES-CIQ", Eq. precond_sqrt and Eq. precond_sqrt_inverse) ----
 *
 * Preconditioner: P = L L^T + sigma^2 I with L the rank-`rank` partial
 * pivoted Cholesky factor of K_XX (greedy pivot: the largest residual
 * diagonal entry, the first index on ties).  msMINRES-CIQ then runs on
 * A = P^{-1/2} K P^{-1/2}, whose spectrum lies in [1, lambda_max(P^{-1}K)]
 * (K_XX - L L^T is positive semidefinite), with the nodes for lambda_min = 1
 * and lambda_max = lmax_margin times the largest Ritz value of a pre-pass on
 * A (or opt->lmin/lmax, opt->quad_w/quad_t for A), and returns
 *     ciq_invsqrt_precond:  out = R' B = P^{-1/2} A^{-1/2} B,  R' R'^T = K^{-1},
 *     ciq_sqrt_precond:     out = R  B = K R' B = P^{1/2} A^{1/2} B,  R R^T = K,
 * square roots of K^{-1} and K that equal the principal ones up to an
 * orthogonal rotation (Eq. precond_sqrt_inverse with P^{1/2} b as the start
 * vector; R = K P^{-1/2} A^{-1/2} of Eq. precond_sqrt).  Convergence follows
 * the conditioning of P^{-1}K instead of K.  The stop rules apply to the
 * estimate in the space of A (relative error of A^{+-1/2} b).  R b has two
 * forms: opt->sqrt_form CIQ_SQRT_MVM is Eq. precond_sqrt as printed, K (R' b)
 * with R' b's solve and stop rule and one more kernel MVM; CIQ_SQRT_IDENTITY
 * (the default) maps A^{1/2} b = (sum w) b - sum_q w_q t_q (A + t_q)^{-1} b
 * with P^{1/2} and needs fewer iterations, but its error in the space of K can
 * be up to sqrt(kappa(P)) times the one the stop rule bounds (measured at
 * N = 8192, sigma^2 = 1e-3: 2e-2 at tol 1e-3, against 2e-4 to 4e-4 for the
 * MVM form at the same tol).  P^{+-1/2}
 * come in closed form from the eigendecomposition of L^T L (host, FP64): with
 * L^T L = U diag(s) U^T and Qh = L U diag(s)^{-1/2},
 * P^{+-1/2} = sigma^{+-1} I + Qh diag((s + sigma^2)^{+-1/2} - sigma^{+-1}) Qh^T,
 * applied in FP32 around every kernel MVM; directions with s <= 1e-10 max(s)
 * are dropped.
 * L: NULL (the factor is computed on the device, rank columns or fewer when
 * the residual diagonal vanishes) or the caller's N x rank factor, column m
 * at L + m * ldl (ldl >= N), host or device, used as given.  1 <= rank <=
 * min(N, 1024); sigma^2 (kern->noise) > 0.  Every other argument, option and
 * return code is that of ciq_sqrt / ciq_invsqrt.  The setup reads L^T L on the host, so these
 * calls synchronise the stream before the iterations as well.
 * info->precond_rank: the directions kept. */
ciq_status ciq_sqrt_precond(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, const float* L,
                            int64_t ldl, const float* B, int T, int Q, double tol, const ciq_options* opt, float* out,
                            ciq_info* info, ciq_stream_t stream);
ciq_status ciq_invsqrt_precond(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, const float* L,
                               int64_t ldl, const float* B, int T, int Q, double tol, const ciq_options* opt,
                               float* out, ciq_info* info, ciq_stream_t stream);

/* The partial pivoted Cholesky factor the preconditioned solves build: L
 * (N x rank, column m at L + m * ldl, ldl >= N; host or device) and the
 * pivots piv[0 .. rank-1] (host or device int64, may be NULL); *rank_out
 * (host, may be NULL) = the columns formed (fewer than rank when the residual
 * diagonal of K_XX - L L^T vanishes first; later columns are 0).  K_XX is
 * evaluated in FP32 (the accurate expf), the residual diagonal and the dot
 * products with earlier columns in FP64.  Synchronous. */
ciq_status ciq_pivoted_cholesky(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, float* L,
                                int64_t ldl, int64_t* piv, int* rank_out, ciq_stream_t stream);

/* Posterior Thompson draws (Sec. 5 "Posterior Sampling for Bayesian
 * Optimization", Eq. thompson_sample): out = mu* + COV*^{1/2} eps at the
 * candidate set Xc (Nc points) given training points Xtr (n points, values
 * y), where
 *     mu*  = m + K*X (K_XX + sigma^2 I)^{-1} (y - m),
 *     COV* = K** - K*X (K_XX + sigma^2 I)^{-1} K_X* + jitter I,
 * for the kernel_type (ciq_kernel_type) with ARD lengthscales
 * (lengthscales[0..d-1], host doubles: coordinate c is divided by
 * lengthscales[c]), outputscale s, noise sigma^2 >= 0 on the training
 * diagonal, jitter > 0 on the candidate diagonal (the paper adds 1e-4) and
 * constant mean m.  COV*^{1/2} is the principal root, by msMINRES-CIQ on COV*
 * (Algorithm "ciq" as in ciq_sqrt, same options, nodes and stop rules; the
 * pre-pass bounds use lambda_min = jitter, a lower bound since
 * K** - K*X M^{-1} K_X* is positive semidefinite).  Every MVM is
 * (K** + jitter I) V on the candidates (on the fly, the opt->precision path)
 * minus C (C^T V) with C = K*X W, W = U diag(lambda^{-1/2}) from the
 * eigendecomposition M = U diag(lambda) U^T of M = K_XX + sigma^2 I (FP64 on the
 * host, directions with lambda <= 1e-13 max(lambda) dropped) and K*X in FP64;
 * C is kept in FP32 (n x round_up(Nc, 128) floats).  Layouts: Xtr n x d,
 * Xc Nc x d row-major; y n floats; eps, out Nc x T as B and out of ciq_sqrt.
 * Host or device pointers.  0 <= n <= CIQ_MAX_TRAIN (n = 0: prior draws,
 * mu* = m); the setup costs O(n^3) on the host and O(n^2 Nc) FP64 on the device.
 * Returns the codes of ciq_sqrt; synchronous. */
ciq_status ciq_posterior_sample(const float* Xtr, int64_t n, const float* y, const float* Xc, int64_t Nc, int d,
                                int kernel_type, const double* lengthscales, double outputscale, double noise,
                                double jitter, double mean, const float* eps, int T, int Q, double tol,
                                const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream);

/* Device workspace bytes a preconditioned solve of this rank needs (for
 * opt->workspace). */
size_t ciq_precond_workspace_bytes(int64_t N, int d, int T, int Q, int rank, const ciq_options* opt);

/* Device workspace bytes a solve with these sizes and options needs. */
size_t ciq_workspace_bytes(int64_t N, int d, int T, int Q, const ciq_options* opt);

/* Allocation-free kernel MVM (the paper has no counterpart: this is a
 * library convenience).  Same result as ciq_kernel_mvm with CIQ_PREC_FP32,
 * out = (K_XX + sigma^2 I) V, for callers that cannot call cudaMalloc --
 * code whose device memory belongs to another allocator, or latency-critical
 * loops where an allocation and the synchronisation it can imply are not
 * allowed.  Its scratch is one static device array of
 * ciq_noalloc_scratch_floats() floats (16 MiB) that every GPU loading the
 * library holds until the process exits; the call needs
 * round_up(round_up(N,128) * round_up(d,4), 64) + T * round_up(N,128) floats
 * of it and returns CIQ_ERR_SCRATCH_TOO_SMALL, touching nothing, when that is
 * more.  X, V, out: device pointers (layouts as above), else CIQ_ERR_ARG.
 * The first call on a device looks up the scratch's device address (once
 * per device, with that device current); make that first call before any
 * stream capture.  The address is kept for the life of the process: after a
 * cudaDeviceReset of a device, do not call this entry point on it again.  All calls share the one array and it keeps the last
 * call's contents (the call clears what must start at zero): calls that
 * overlap on the GPU, e.g. on two streams, race on it.  Allocates nothing
 * (no cudaMalloc, cudaFree or allocating library routine).  Asynchronous on
 * stream. */
ciq_status ciq_kernel_mvm_noalloc(const float* X, int64_t N, int d, const ciq_kernel* kern,
                                  const float* V, int T, float* out, ciq_stream_t stream);

/* Size in floats of the static scratch behind ciq_kernel_mvm_noalloc. */
size_t ciq_noalloc_scratch_floats(void);

#ifdef __cplusplus
}
#endif
#endif /* CIQ_H */
