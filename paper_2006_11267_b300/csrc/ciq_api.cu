// C entry points of libciq (include/ciq.h): argument checks, workspace
// layout, and the launch sequence of msMINRES-CIQ (Algorithm "ciq"):
//
//   points -> [Lanczos pre-pass -> Ritz extremes -> bounds -> nodes]  (device)
//          -> init (q_1 = b/||b||) -> J x (kernel MVM + msMINRES step)   (device)
//          -> combine (K^{-1/2} b or K^{1/2} b) -> summary               (device)
//
// The host only launches: it reads one device flag ("every column stopped")
// per batch of `check_every` iterations, one batch behind the launches, so
// the GPU never waits on the host.
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "batched.cuh"
#include "host_checks.cuh"
#include "krylov.cuh"
#include "mlp.cuh"
#include "mvm_stored.cuh"
#include "mvm_tc.cuh"
#include "posterior.cuh"
#include "precond.cuh"
#include "spectral.cuh"
#include "symeig.h"

using namespace ciq;

namespace {

constexpr size_t kAlign = 256;

struct Arena {
    char* base = nullptr;
    size_t off = 0;
    template <typename T>
    T* take(size_t n) {
        off = (off + kAlign - 1) / kAlign * kAlign;
        T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
        off += n * sizeof(T);
        return p;
    }
};

// Row chunks per column of the recurrence (its grid is chunks x T blocks):
// the grid should fill whole waves of resident blocks, so among one to three
// waves the chunk count with the best fill is taken (a further wave only for
// at least 2 % more fill; every block also re-reads its column's partial
// sums), at most Npad / 1024 chunks.
void choose_chunks(int64_t Npad, int T, int* nchunks, int64_t* rpc) {
    const int64_t max_chunks = std::max<int64_t>(1, Npad / 1024);
    const int64_t W = step_blocks_per_wave();
    int64_t ch = 1;
    double best_fill = -1.0;
    for (int64_t m = 1; m <= 3; ++m) {
        const int64_t c = std::min<int64_t>(std::max<int64_t>(1, m * W / T), max_chunks);
        const int64_t blocks = c * T;
        const double fill = (double)blocks / (double)(((blocks + W - 1) / W) * W);
        if (fill > best_fill + 0.02) { best_fill = fill; ch = c; }
    }
    const int64_t r = round_up((Npad + ch - 1) / ch, kRowPad);
    *rpc = r;
    *nchunks = (int)((Npad + r - 1) / r);
}

ciq_status from_cuda(cudaError_t e) {
    if (e == cudaSuccess) return CIQ_OK;
    if (e == cudaErrorMemoryAllocation) return CIQ_ERR_NOMEM;
    return CIQ_ERR_CUDA;
}

#define CIQ_TRY(...)                                    \
    do {                                                \
        cudaError_t _e = (__VA_ARGS__);                 \
        if (_e != cudaSuccess) { rc = from_cuda(_e); goto done; } \
    } while (0)

bool valid_options(const ciq_options& o) {
    return !(o.max_iter < 1 || o.max_iter > 1000000 || o.lanczos_iters < 1 || o.lanczos_iters > 512 ||
             o.check_every < 1 || !(o.lmax_margin >= 1.0) || !(o.lmin_div >= 1.0) ||
             (o.stop_rule != CIQ_STOP_RESIDUAL && o.stop_rule != CIQ_STOP_ERRBOUND) ||
             (o.sqrt_form != CIQ_SQRT_IDENTITY && o.sqrt_form != CIQ_SQRT_MVM) ||
             (o.precision < CIQ_PREC_FP32 || o.precision > CIQ_PREC_FP16) ||
             (o.mvm < CIQ_MVM_AUTO || o.mvm > CIQ_MVM_STORED) || o.tc_split < 0 || o.tc_split > 8 ||
             o.fault_inject < 0 || o.fault_inject > 1 || o.krylov < CIQ_KRYLOV_AUTO ||
             o.krylov > CIQ_KRYLOV_BASIS || o.batch_split_rows < 0 ||
             (o.batch_split_rows > 0 && (o.batch_split < 1 || o.batch_split > 8)) || o.precond_rank < 0 ||
             o.precond_rank > kPcMaxRank);
}

// Pinned host words for the convergence flag, one set per host thread.
int* pinned_flags() {
    thread_local int* p = nullptr;
    if (!p) {
        if (cudaHostAlloc(reinterpret_cast<void**>(&p), 4 * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    return p;
}

void keep_pool_warm() {
    static bool done = false;
    if (done) return;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return; }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    done = true;
}

// ---------------------------------------------------------------- plan ----
template <typename R>
struct Plan {
    int64_t N, Npad;
    int d, dp, T, Q;
    int jmax, JL;
    int nparts, nparts1, nchunks, nchunks1;
    int64_t rpc, rpc1;
    bool tc;                      // tensor-core MVM
    bool stored;                  // stored-K MVM (K formed once, Npad x Npad)
    float kscale = 1.f;           // stored K on tensor cores: power-of-two scale of K
    int precision;
    bool stage_x, stage_b, stage_out, stage_start;
    bool prepass;
    bool tri_on = false;          // record column 0's msMINRES tridiagonal
    int tc_max_split = 8;         // CTAs per row tile of the tensor-core MVM (batches: 1)
    int fault_inject = 0;         // ciq_options.fault_inject (testing the bounded-wait path)
    bool basis = false;           // stored-basis form (CIQ_KRYLOV_BASIS)
    bool pair_p = false;          // a solve: keeps p as a float pair where the MVM runs on CUDA cores
    bool vjp = false;             // backward pass: T = 2 T_B columns [B | G], basis form
    int pc_rank = 0;              // pivoted-Cholesky preconditioner rank (0: none)
    int lr_rank = -1;             // low-rank correction -C C^T of the MVM (>= 0: on)
    float *lr_g = nullptr, *lr_s = nullptr;   // its g = -1 and reduction scratch
    bool stage_l = false;         // the caller's factor L is on the host
    // pointers (valid once an arena base is set)
    R *Xp, *QA, *QB, *Y, *Ylo, *Bw, *D, *LA, *LB, *V, *sco;
    double *rcoef, *gauss, *bco, *ycoef, *vpart, *vgrad;
    float* Xq;
    R *sx, *sb, *sout, *sstart;
    R* plo = nullptr;                 // trailing part of the Lanczos p (FP32 CUDA-core basis solves)
    float* Kst;
    double *partials, *ynp, *beta, *beta1, *giv, *phifinal, *nodes, *summary, *tri;
    double *lpart, *lynp, *bpar, *lalpha, *lbeta;
    int *status, *iters, *brk, *cnt, *all_done, *jeff, *ldone;
    TcPoints tcp;
    // Preconditioner: factor L and basis Qh [pc_rank][Npad], g^-/g^+, the
    // scratch of its applications, the MVM's input P^{-1/2} q and raw output
    // K P^{-1/2} q, the A-space result, and the setup scratch.
    float *Lf = nullptr, *Qh = nullptr, *pc_g = nullptr, *pcs = nullptr, *Up = nullptr, *Op = nullptr,
          *Apre = nullptr, *sL = nullptr;
    double *dres = nullptr, *Gm = nullptr, *gpart = nullptr, *Wm = nullptr;
    int *piv = nullptr, *rank_out = nullptr;
    void* cwork = nullptr;
    size_t bytes;

    void layout(char* base) {
        Arena a;
        a.base = base;
        Xp = a.take<R>((size_t)Npad * dp);
        if (basis) {
            // q_0 = 0 in slot 0, q_1 in slot 1: the first two slots double as QB, QA.
            V = a.take<R>(((size_t)jmax + 2) * T * Npad);
            QB = V;
            QA = base ? V + (size_t)T * Npad : nullptr;
        } else {
            V = nullptr;
            QA = a.take<R>((size_t)T * Npad);
            QB = a.take<R>((size_t)T * Npad);
        }
        Y = a.take<R>((size_t)T * Npad);
        Ylo = a.take<R>((size_t)T * Npad);
        Bw = a.take<R>((size_t)T * Npad);
        D = basis ? nullptr : a.take<R>((size_t)2 * Q * T * Npad);
        // FP32 CUDA-core solves keep p as a float pair (both Krylov forms, batched too).
        plo = (pair_p && !tc && !stored && sizeof(R) == 4 && pc_rank <= 0 && lr_rank < 0)
                  ? a.take<R>((size_t)T * Npad) : nullptr;
        rcoef = basis ? a.take<double>((size_t)jmax * Q * T * 4) : nullptr;
        gauss = basis ? a.take<double>((size_t)2 * T * 4) : nullptr;
        bco = basis ? a.take<double>(((size_t)jmax + 1) * T) : nullptr;
        sco = a.take<R>((size_t)T * kScoStride);
        ycoef = vjp ? a.take<double>(((size_t)jmax + 1) * Q * T) : nullptr;
        Xq = vjp ? a.take<float>((size_t)Q * T * Npad) : nullptr;
        vpart = vjp ? a.take<double>((size_t)vjp_partials(Npad, T / 2, Q)) : nullptr;
        vgrad = vjp ? a.take<double>(3) : nullptr;
        partials = a.take<double>((size_t)nparts * T * 3);
        ynp = a.take<double>((size_t)2 * nchunks * T);
        beta = a.take<double>((size_t)2 * T);
        beta1 = a.take<double>((size_t)T);
        giv = a.take<double>((size_t)2 * Q * T * 5);
        phifinal = a.take<double>((size_t)Q * T);
        nodes = a.take<double>(kNodeCount);
        summary = a.take<double>(8);
        status = a.take<int>(T);
        iters = a.take<int>(T);
        brk = a.take<int>(T);
        cnt = a.take<int>((size_t)jmax + 2);
        all_done = a.take<int>(1);
        tri = tri_on ? a.take<double>(2 * (size_t)jmax + 3) : nullptr;
        if (prepass) {
            LA = a.take<R>((size_t)Npad);
            LB = a.take<R>((size_t)Npad);
            lpart = a.take<double>((size_t)nparts1 * 3);
            lynp = a.take<double>((size_t)nchunks1);
            bpar = a.take<double>(2);
            lalpha = a.take<double>((size_t)JL);
            lbeta = a.take<double>((size_t)JL + 1);
            jeff = a.take<int>(1);
            ldone = a.take<int>(1);
        } else {
            LA = LB = nullptr; lpart = lynp = bpar = lalpha = lbeta = nullptr; jeff = ldone = nullptr;
        }
        sx = stage_x ? a.take<R>((size_t)N * d) : nullptr;
        sb = stage_b ? a.take<R>((size_t)N * T) : nullptr;
        sout = stage_out ? a.take<R>((size_t)N * T) : nullptr;
        sstart = stage_start ? a.take<R>((size_t)N) : nullptr;
        if (tc) {
            char* q = a.take<char>(tc_points_bytes(Npad, T, tc_max_split));
            tcp = tc_points_layout(q, Npad, T, precision, tc_max_split, d);
            tcp.inject = fault_inject;
        }
        Kst = stored ? a.take<float>((size_t)Npad * Npad) : nullptr;
        if (lr_rank >= 0) {
            const int rk = std::max(lr_rank, 1);
            lr_g = a.take<float>((size_t)rk);
            lr_s = a.take<float>(pc_scratch_floats(Npad, rk, T));
            if (pc_rank <= 0) Op = a.take<float>((size_t)T * Npad);
        }
        if (pc_rank > 0) {
            const size_t RK = (size_t)pc_rank;
            Lf = a.take<float>(RK * Npad);
            Qh = a.take<float>(RK * Npad);
            pc_g = a.take<float>(2 * RK);
            pcs = a.take<float>(pc_scratch_floats(Npad, pc_rank, T));
            Up = a.take<float>((size_t)T * Npad);
            Op = a.take<float>((size_t)T * Npad);
            Apre = a.take<float>((size_t)T * Npad);
            dres = a.take<double>((size_t)Npad);
            Gm = a.take<double>(RK * RK);
            gpart = a.take<double>((size_t)pc_gram_scratch(Npad, pc_rank));
            Wm = a.take<double>(RK * RK);
            piv = a.take<int>(RK + 1);
            rank_out = a.take<int>(1);
            cwork = a.take<char>(pc_cholesky_work_bytes(Npad));
            sL = stage_l ? a.take<float>(RK * (size_t)N) : nullptr;
        }
        bytes = a.off + kAlign;
    }
};

// Largest stored basis the AUTO form takes: a quarter of the device memory,
// at most 64 GiB (64 GiB when no device answers).
size_t basis_cap_bytes() {
    const size_t cap = (size_t)64 << 30;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return cap; }
    return std::min(cap, tot / 4);
}

// Stored-basis form of a single solve (batched solves always recur).
bool use_basis(const ciq_options& o, size_t elem, int64_t Npad, int T) {
    if (o.krylov == CIQ_KRYLOV_RECURRENCE) return false;
    if (o.krylov == CIQ_KRYLOV_BASIS) return true;
    const size_t bytes = ((size_t)o.max_iter + 2) * (size_t)T * (size_t)Npad * elem;
    return elem == 4 && bytes <= basis_cap_bytes();
}

template <typename R>
Plan<R> make_plan(int64_t N, int d, int T, int Q, const ciq_options& o, bool prepass, bool tc,
                  bool allow_basis = false) {
    Plan<R> p{};
    p.precision = o.precision;
    p.N = N;
    p.d = d;
    p.dp = dim_pad(d);
    p.Npad = round_up(N, kRowPad);
    p.T = T;
    p.Q = Q;
    p.jmax = o.max_iter;
    p.JL = o.lanczos_iters;
    p.tc = tc;
    p.tc_max_split = o.tc_split > 0 ? o.tc_split : 8;
    p.fault_inject = o.fault_inject;
    p.stored = sizeof(R) == 4 && o.mvm == CIQ_MVM_STORED;
    p.nparts = tc ? (int)tc_row_tiles(p.Npad)
                  : p.stored ? (int)stored_row_tiles(p.Npad, T) : (int)mvm_simt_row_tiles<R>(p.Npad, T);
    // The pre-pass (one column) runs on the solve's MVM path: tensor cores,
    // stored K or CUDA cores.
    p.nparts1 = tc ? (int)tc_row_tiles(p.Npad)
                   : p.stored ? (int)stored_row_tiles(p.Npad, 1) : (int)mvm_simt_row_tiles<R>(p.Npad, 1);
    choose_chunks(p.Npad, T, &p.nchunks, &p.rpc);
    choose_chunks(p.Npad, 1, &p.nchunks1, &p.rpc1);
    p.prepass = prepass;
    p.basis = allow_basis && use_basis(o, sizeof(R), p.Npad, T);
    p.pair_p = allow_basis;
    p.layout(nullptr);
    return p;
}

template <typename R>
KrylovState<R> krylov_state(const Plan<R>& p, int op, const ciq_options& o, double tol) {
    KrylovState<R> s{};
    s.N = p.N; s.Npad = p.Npad; s.T = p.T; s.Q = p.Q;
    s.nparts = p.nparts; s.nchunks = p.nchunks; s.rows_per_chunk = p.rpc;
    s.QA = p.QA; s.QB = p.QB; s.D = p.D; s.Y = p.Y; s.Ylo = p.Ylo; s.Bw = p.Bw;
    s.partials = p.partials; s.ynp = p.ynp; s.beta = p.beta; s.beta1 = p.beta1;
    s.giv = p.giv; s.phifinal = p.phifinal; s.status = p.status; s.iters = p.iters;
    s.brk = p.brk; s.cnt = p.cnt; s.all_done = p.all_done; s.nodes = p.nodes;
    s.summary = p.summary; s.tri = p.tri; s.jmax = p.jmax; s.op = op; s.stop_rule = o.stop_rule; s.tol = tol;
    s.basis = p.V; s.rcoef = p.rcoef; s.gauss = p.gauss; s.bco = p.bco; s.sco = p.sco; s.ycoef = p.ycoef;
    s.plo = p.plo;
    s.breakdown_rtol = sizeof(R) == 4 ? 1e-6 : 1e-13;
    return s;
}

template <typename R>
LanczosState<R> lanczos_state(const Plan<R>& p) {
    LanczosState<R> s{};
    s.N = p.N; s.Npad = p.Npad; s.nparts = p.nparts1; s.nchunks = p.nchunks1;
    s.rows_per_chunk = p.rpc1; s.iters = p.JL;
    s.LA = p.LA; s.LB = p.LB; s.partials = p.lpart; s.ynp = p.lynp; s.bpar = p.bpar;
    s.alpha = p.lalpha; s.beta = p.lbeta; s.jeff = p.jeff; s.done = p.ldone;
    return s;
}

template <typename R>
MvmArgs<R> mvm_args(const Plan<R>& p, const ciq_kernel& k) {
    MvmArgs<R> a{};
    a.X = p.Xp; a.N = p.N; a.Npad = p.Npad; a.dp = p.dp; a.kt = k.type;
    a.s = (R)k.outputscale; a.noise = (R)k.noise; a.ldv = p.Npad;
    return a;
}

template <typename R>
cudaError_t launch_mvm(const Plan<R>& p, const MvmArgs<R>& a, bool unit_columns, cudaStream_t st,
                       bool scale_ready = false);

// The MVM of the preconditioned operator A = P^{-1/2} K P^{-1/2} with the
// Lanczos epilogue of `a`: U = P^{-1/2} q, O' = K U (plain MVM), then
// p = P^{-1/2} O' - beta q_prev and the partial sums.
template <typename R>
cudaError_t precond_mvm(const Plan<R>& p, const PrecondState& pc, const MvmArgs<R>& a, cudaStream_t st,
                        bool scale_ready = false, const PrecondState* lr = nullptr) {
    if constexpr (sizeof(R) == 4) {
        if (pc.lowrank) {
            // (K - C C^T) q: the plain MVM of the unit columns q, then the
            // correction and the Lanczos epilogue.
            MvmArgs<R> m = a;
            m.mode = kPlain;
            m.out = p.Op;
            m.ldo = p.Npad;
            m.lz_q = nullptr;
            m.lz_sco = nullptr;
            cudaError_t e = launch_mvm(p, m, true, st, scale_ready);
            if (e != cudaSuccess) return e;
            return launch_lowrank_lanczos(pc, a.V, p.Op, a.V, a.qprev, a.pout, a.beta, a.partials, a.T, a.stop, st);
        }
        // On tensor cores the operand scales of U come from the reduction of
        // P^{-1/2} (the columns of q have norm 1), so the MVM skips its own pass.
        cudaError_t e = launch_pc_apply(pc, a.V, p.Npad, a.T, true, p.Up, p.Npad, a.stop, st,
                                        p.tc ? p.tcp.vscale : nullptr, p.tc ? p.tcp.TP : 0);
        if (e != cudaSuccess) return e;
        MvmArgs<R> m = a;
        m.mode = kPlain;
        m.V = p.Up;
        m.out = p.Op;
        m.ldo = p.Npad;
        m.lz_q = nullptr;
        m.lz_sco = nullptr;
        e = launch_mvm(p, m, p.tc, st, p.tc);
        if (e != cudaSuccess) return e;
        // A low-rank term under the preconditioner (posterior covariance):
        // O' = K U - C C^T U before the second application of P^{-1/2}.
        if (lr && (e = launch_lowrank_apply(*lr, p.Up, p.Op, a.T, a.stop, st)) != cudaSuccess) return e;
        return launch_pc_lanczos(pc, p.Op, a.V, a.qprev, a.pout, a.beta, a.partials, a.T, a.stop, st);
    }
    return cudaErrorNotSupported;
}

// Lanczos pre-pass on the device; leaves nodes in p.nodes.  With a
// preconditioner the pre-pass runs on A and lambda_min = 1 (P <= K).
template <typename R>
cudaError_t run_prepass(const Plan<R>& p, const ciq_kernel& k, const ciq_options& o, int Q,
                        const R* start_dev, cudaStream_t st, const PrecondState* pc = nullptr,
                        const PrecondState* lr = nullptr) {
    LanczosState<R> ls = lanczos_state(p);
    cudaError_t e = launch_lanczos_init(ls, start_dev, o.seed, st);
    if (e != cudaSuccess) return e;
    MvmArgs<R> a = mvm_args(p, k);
    a.T = 1;
    a.mode = kLanczos;
    a.partials = p.lpart;
    a.stop = p.ldone;
    for (int j = 1; j <= p.JL; ++j) {
        a.V = (j & 1) ? p.LA : p.LB;
        a.qprev = (j & 1) ? p.LB : p.LA;
        a.beta = p.bpar + (j & 1);
        if (pc) e = precond_mvm(p, *pc, a, st, false, lr);
        else e = (p.stored || p.tc) ? launch_mvm(p, a, true, st) : launch_mvm_simt(a, st);
        if (e != cudaSuccess) return e;
        if ((e = launch_lanczos_step(ls, j, st)) != cudaSuccess) return e;
    }
    return launch_bounds_nodes(ls, p.nodes, Q, pc && !pc->lowrank ? 1.0 : k.noise, o.lmax_margin, o.lmin_div, st);
}

template <typename R>
cudaError_t tc_prepare(const Plan<R>& p, int kt, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (p.tc) return launch_tc_prepare(p.tcp, p.Xp, p.N, p.dp, p.d, kt, st);
    }
    return cudaSuccess;
}

// unit_columns: V's columns have norm 1 (Lanczos vectors), which fixes the
// power-of-two operand scale of the tensor-core MVM.
template <typename R>
cudaError_t launch_mvm(const Plan<R>& p, const MvmArgs<R>& a, bool unit_columns, cudaStream_t st,
                       bool scale_ready) {
    if constexpr (sizeof(R) == 4) {
        if (p.stored && p.tc)
            return launch_stored_mvm_tc(p.Kst, p.Npad, p.tcp, a, p.kscale, unit_columns, st, scale_ready);
        if (p.tc) return launch_mvm_tc(p.tcp, a, unit_columns, st, scale_ready);
        if (p.stored) return launch_stored_mvm(p.Kst, p.Npad, a, st);
    }
    return launch_mvm_simt(a, st);
}

// Form the stored K once (stored-K mode only).
template <typename R>
cudaError_t form_stored(const Plan<R>& p, const ciq_kernel& k, cudaStream_t st) {
    if constexpr (sizeof(R) == 4) {
        if (p.stored)
            return launch_kernel_matrix(p.Xp, p.N, p.Npad, p.dp, k.type, (float)k.outputscale, (float)k.noise, p.Kst,
                                        p.Npad, p.Npad, st);
    }
    return cudaSuccess;
}

// CUDA events of the profile mode: one event between consecutive launches of
// a batch of iterations, harvested one batch behind like the convergence flag.
struct Profile {
    bool on = false;
    cudaEvent_t t_start = nullptr, t_pre0 = nullptr, t_pre1 = nullptr, t_loop = nullptr,
                t_loop_end = nullptr, t_end = nullptr;
    std::vector<cudaEvent_t> ev[2];
    std::vector<double> mvm_ms, step_ms;
    cudaError_t create() {
        cudaEvent_t* all[] = {&t_start, &t_pre0, &t_pre1, &t_loop, &t_loop_end, &t_end};
        for (auto* e : all) {
            cudaError_t r = cudaEventCreate(e);
            if (r != cudaSuccess) return r;
        }
        return cudaSuccess;
    }
    void destroy() {
        cudaEvent_t all[] = {t_start, t_pre0, t_pre1, t_loop, t_loop_end, t_end};
        for (auto e : all)
            if (e) cudaEventDestroy(e);
        for (auto& v : ev)
            for (auto e : v)
                if (e) cudaEventDestroy(e);
    }
};

// A preconditioned solve's factor: the caller's L (N x rank, column m at
// L + m * ldl, host or device) or, when L is null, the pivoted Cholesky of
// K_XX computed here.
struct PcSpec {
    const float* L;
    int64_t ldl;
    int rank;
};

// A low-rank correction of the MVM, (K - C C^T) V, with C^T given on the
// device as [rank][Npad] (the posterior covariance K** - K*X M^{-1} K_X* of
// a draw, C = K*X M^{-1/2}); mu (device, Npad floats, may be null) is added
// to every output column.
struct LrSpec {
    const float* Ct;
    int rank;
    const float* mu;
};

// Preconditioner setup (App. "Preconditioning msMINRES-CIQ"): the factor,
// G = L^T L on the device, its eigendecomposition on the host, the basis
// Qh = L U diag(s)^{-1/2} of the directions with s > 1e-10 max(s) and the
// coefficients of P^{+-1/2}.  Synchronises the stream (the host reads G).
ciq_status build_precond(const Plan<float>& p, const ciq_kernel& k, const PcSpec& spec, const float* Ld,
                         cudaStream_t st, PrecondState* pc, int* launches, const float* Ct = nullptr, int rk = 0) {
    int R = spec.rank;
    cudaError_t e = cudaSuccess;
    if (Ld) {
        e = cudaMemsetAsync(p.Lf, 0, sizeof(float) * (size_t)R * p.Npad, st);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(p.Lf, sizeof(float) * p.Npad, Ld, sizeof(float) * spec.ldl, sizeof(float) * p.N, R,
                                  cudaMemcpyDeviceToDevice, st);
    } else {
        e = launch_pivoted_cholesky(p.Xp, p.N, p.Npad, p.dp, k.type, (float)k.outputscale, R, p.Lf, p.piv, p.dres,
                                    p.cwork, p.rank_out, st, Ct, rk);
        *launches += R + 1 + (rk > 0 ? 1 : 0);
        int rr = R;
        if (e == cudaSuccess) e = cudaMemcpyAsync(&rr, p.rank_out, sizeof(int), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        R = std::min(R, std::max(0, rr));
    }
    if (e != cudaSuccess) return from_cuda(e);
    const double sig2 = k.noise, sig = std::sqrt(k.noise);
    std::vector<double> G((size_t)R * R), w(R), Z((size_t)R * R), W;
    std::vector<float> g;
    int Rk = 0;
    if (R > 0) {
        e = launch_gram(p.Lf, p.Npad, R, p.gpart, p.Gm, st);
        *launches += 2;
        if (e == cudaSuccess) e = cudaMemcpyAsync(G.data(), p.Gm, sizeof(double) * G.size(), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return from_cuda(e);
        for (double x : G)
            if (!std::isfinite(x)) return CIQ_ERR_NAN;
        if (!symeig::eigh(R, G.data(), w.data(), Z.data())) return CIQ_ERR_NAN;
        const double smax = w[R - 1];
        std::vector<int> keep;
        for (int c = 0; c < R; ++c)
            if (w[c] > 1e-10 * smax && w[c] > 0.0) keep.push_back(c);
        Rk = (int)keep.size();
        W.assign((size_t)R * std::max(Rk, 1), 0.0);
        g.assign(2 * (size_t)std::max(Rk, 1), 0.f);
        for (int c = 0; c < Rk; ++c) {
            const double sv = w[keep[c]], inv = 1.0 / std::sqrt(sv), root = std::sqrt(sv + sig2);
            for (int m = 0; m < R; ++m) W[(size_t)m + (size_t)c * R] = Z[(size_t)m + (size_t)keep[c] * R] * inv;
            g[c] = (float)(1.0 / root - 1.0 / sig);                  // g^-
            g[Rk + c] = (float)(root - sig);                         // g^+
        }
        if (Rk > 0) {
            e = cudaMemcpyAsync(p.Wm, W.data(), sizeof(double) * (size_t)R * Rk, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(p.pc_g, g.data(), sizeof(float) * 2 * (size_t)Rk, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = launch_basis_from_factor(p.Lf, p.Npad, R, p.Wm, Rk, p.Qh, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);     // the host vectors go out of scope
            *launches += 1;
            if (e != cudaSuccess) return from_cuda(e);
        }
    }
    PrecondState s;
    s.N = p.N;
    s.Npad = p.Npad;
    s.rank = Rk;
    s.Qh = p.Qh;
    s.gm = p.pc_g;
    s.gp = p.pc_g + Rk;
    s.sigma = (float)sig;
    s.inv_sigma = (float)(1.0 / sig);
    s.cpart = p.pcs;
    s.coef = p.pcs + (pc_scratch_floats(p.Npad, p.pc_rank, p.T) - (size_t)Rk * p.T);
    s.T = p.T;
    *pc = s;
    return CIQ_OK;
}

// Kd: a caller's explicit matrix (N x N, leading dimension ldk) instead of X
// and a kernel; the solve then runs on the stored-K MVM with no noise term.
template <typename R>
ciq_status solve(const R* X, int64_t N, int d, const ciq_kernel* kern, const R* B, int T, int Q,
                 double tol, const ciq_options* opt, R* out, ciq_info* info, cudaStream_t st,
                 int op, bool fp64, const float* Kd = nullptr, int64_t ldk = 0, double* vjp_grad = nullptr,
                 const PcSpec* pcs = nullptr, const LrSpec* lrs = nullptr) {
    // A low-rank term may sit under a preconditioner that the device factors (no caller's L).
    if (lrs && (fp64 || Kd || vjp_grad || (pcs && pcs->L) || lrs->rank < 0 || (lrs->rank > 0 && !lrs->Ct)))
        return CIQ_ERR_ARG;
    const bool dense = Kd != nullptr;
    const bool vjp = vjp_grad != nullptr;
    if (pcs) {
        // Preconditioned solves: FP32 vectors, kernel MVMs, identity forms only.
        if (fp64 || dense || vjp || pcs->rank < 1 || pcs->rank > kPcMaxRank || pcs->rank > N ||
            (pcs->L && pcs->ldl < N) || !kern || !(kern->noise > 0.0))
            return CIQ_ERR_ARG;
    }
    if ((!dense && !X) || !B || !out || N < 1 || d < 1 || d > CIQ_MAX_DIM || T < 1 || Q < 1 || Q > CIQ_MAX_Q ||
        !(tol >= 0.0) || !valid_kernel(kern) || (dense && (ldk < N || fp64)))
        return CIQ_ERR_ARG;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    if (!valid_options(o)) return CIQ_ERR_ARG;
    if (dense) {
        if (o.precision != CIQ_PREC_FP32) return CIQ_ERR_UNSUPPORTED;
        o.mvm = CIQ_MVM_STORED;
    }
    if (vjp) {
        // The backward pass needs every shift's solution: the stored-basis form.
        if (fp64 || dense || T % 2 != 0 || o.krylov == CIQ_KRYLOV_RECURRENCE ||
            (op == kOpSqrtIdentity && o.sqrt_form == CIQ_SQRT_MVM))
            return CIQ_ERR_UNSUPPORTED;
        o.krylov = CIQ_KRYLOV_BASIS;
    }
    if ((o.quad_w == nullptr) != (o.quad_t == nullptr)) return CIQ_ERR_ARG;
    if (o.mvm == CIQ_MVM_STORED && !fp64 && o.precision == CIQ_PREC_TF32) return CIQ_ERR_UNSUPPORTED;
    bool tc = false;
    if (!fp64 && o.precision != CIQ_PREC_FP32) {
        if (!tc_supported(o.precision, d) || tc_padded_t(T) < 0) return CIQ_ERR_UNSUPPORTED;
        tc = true;
    }
    if (op == kOpSqrtIdentity && o.sqrt_form == CIQ_SQRT_MVM) op = kOpSqrtMvm;
    // Preconditioned literal form R b = K (R' b) (Eq. precond_sqrt as printed):
    // the solve, its stop rule and its combine are those of R' b.
    const bool pc_literal = pcs && op == kOpSqrtMvm;
    if (pc_literal) op = kOpInvSqrt;
    const bool given_nodes = o.quad_w != nullptr;
    const bool given_bounds = !given_nodes && o.lmin > 0.0 && o.lmax > 0.0;
    if (given_bounds && !(o.lmax >= o.lmin)) return CIQ_ERR_ARG;
    double hw[CIQ_MAX_Q] = {0}, ht[CIQ_MAX_Q] = {0};
    if (given_nodes) {
        for (int q = 0; q < Q; ++q) {
            hw[q] = o.quad_w[q];
            ht[q] = o.quad_t[q];
            if (!(ht[q] >= 0.0) || !std::isfinite(hw[q]) || !std::isfinite(ht[q])) return CIQ_ERR_ARG;
        }
    }
    const bool prepass = !given_nodes && !given_bounds;
    keep_pool_warm();

    Plan<R> p = make_plan<R>(N, d, T, Q, o, prepass, tc, true);
    p.vjp = vjp;
    // Stored K on tensor cores: max_i K_ii = outputscale + sigma^2 sets K's scale.
    if (p.stored && p.tc) p.kscale = stored_tc_scale(kern->outputscale + kern->noise);
    if (pcs) {
        p.pc_rank = pcs->rank;
        p.stage_l = pcs->L && !device_accessible(pcs->L);
        p.nparts = p.nparts1 = (int)pc_row_tiles(p.Npad);    // the preconditioned epilogue's row tiles
    }
    if (lrs) {
        p.lr_rank = lrs->rank;
        p.nparts = p.nparts1 = (int)pc_row_tiles(p.Npad);
    }
    p.stage_x = !dense && !device_accessible(X);
    p.stage_b = !device_accessible(B);
    p.stage_out = !device_accessible(out);
    p.stage_start = prepass && o.lanczos_start && !device_accessible(o.lanczos_start);
    p.layout(nullptr);
    const size_t need = p.bytes;
    char* base = nullptr;
    bool owned = false;
    ciq_status rc = CIQ_OK;
    int* flags = pinned_flags();
    double summary[8] = {0};
    int tc_timeout = 0;                // the tensor-core MVM's error flag (a bounded wait gave up)
    double nodes[kNodeCount] = {0};
    int last_j = 0;
    int launches = 0;
    PrecondState pcst;
    PrecondState lrst;                 // the low-rank term when it sits under a preconditioner
    bool pc_on = false, lr_under_pc = false;
    cudaEvent_t ev[2] = {nullptr, nullptr};
    Profile prof;
    prof.on = o.profile != 0;
    if (!flags) return CIQ_ERR_CUDA;
    if (prof.on && prof.create() != cudaSuccess) { cudaGetLastError(); return CIQ_ERR_CUDA; }
    if (o.workspace) {
        if (o.workspace_bytes < need) return CIQ_ERR_ARG;
        base = static_cast<char*>(o.workspace);
    } else {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), need, st);
        if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? CIQ_ERR_NOMEM : CIQ_ERR_CUDA; }
        owned = true;
    }
    {
        p.layout(base);
        const R* Xd = X;
        const R* Bd = B;
        R* outd = out;
        const R* startd = reinterpret_cast<const R*>(o.lanczos_start);
        if (p.stage_x) {
            CIQ_TRY(cudaMemcpyAsync(p.sx, X, sizeof(R) * (size_t)N * d, cudaMemcpyHostToDevice, st));
            Xd = p.sx;
        }
        if (p.stage_b) {
            CIQ_TRY(cudaMemcpyAsync(p.sb, B, sizeof(R) * (size_t)N * T, cudaMemcpyHostToDevice, st));
            Bd = p.sb;
        }
        if (p.stage_out) outd = p.sout;
        if (p.stage_start) {
            CIQ_TRY(cudaMemcpyAsync(p.sstart, o.lanczos_start, sizeof(R) * (size_t)N, cudaMemcpyHostToDevice, st));
            startd = p.sstart;
        }
        CIQ_TRY(cudaMemsetAsync(p.cnt, 0, sizeof(int) * ((size_t)p.jmax + 2), st));
        CIQ_TRY(cudaMemsetAsync(p.all_done, 0, sizeof(int), st));
        if (p.basis) CIQ_TRY(cudaMemsetAsync(p.gauss, 0, sizeof(double) * 2 * 4 * (size_t)T, st));
        if (prof.on) CIQ_TRY(cudaEventRecord(prof.t_start, st));
        if (dense) {
            // The caller's matrix into the zero-padded Npad x Npad layout.
            CIQ_TRY(cudaMemsetAsync(p.Kst, 0, sizeof(float) * (size_t)p.Npad * p.Npad, st));
            CIQ_TRY(cudaMemcpy2DAsync(p.Kst, sizeof(float) * p.Npad, Kd, sizeof(float) * ldk, sizeof(float) * N, N,
                                      cudaMemcpyDefault, st));
            CIQ_TRY(cudaMemsetAsync(p.Xp, 0, sizeof(R) * (size_t)p.Npad * p.dp, st));
        } else {
            CIQ_TRY(launch_prepare_points<R, R>(Xd, N, d, p.Npad, p.dp, 1.0 / kern->lengthscale, p.Xp, st));
            CIQ_TRY(tc_prepare(p, kern->type, st));
            CIQ_TRY(form_stored(p, *kern, st));
            launches += p.stored ? 1 : 0;
        }
        if constexpr (sizeof(R) == 4) {
            if (lrs) {
                std::vector<float> neg((size_t)std::max(lrs->rank, 1), -1.f);
                CIQ_TRY(cudaMemcpyAsync(p.lr_g, neg.data(), sizeof(float) * neg.size(), cudaMemcpyHostToDevice, st));
                CIQ_TRY(cudaStreamSynchronize(st));
                PrecondState l;
                l.N = N;
                l.Npad = p.Npad;
                l.rank = lrs->rank;
                l.Qh = lrs->Ct;
                l.gm = p.lr_g;
                l.gp = p.lr_g;
                l.sigma = 1.f;
                l.inv_sigma = 1.f;
                l.cpart = p.lr_s;
                l.coef = p.lr_s + (pc_scratch_floats(p.Npad, std::max(lrs->rank, 1), T) -
                                   (size_t)std::max(lrs->rank, 1) * T);
                l.T = T;
                l.lowrank = true;
                l.mu = lrs->mu;
                if (p.pc_rank > 0) {
                    lrst = l;
                    lr_under_pc = true;
                } else {
                    pcst = l;
                    pc_on = true;
                }
            }
            if (p.pc_rank > 0) {
                const float* Ld = pcs->L;
                if (p.stage_l) {
                    CIQ_TRY(cudaMemcpy2DAsync(p.sL, sizeof(float) * N, pcs->L, sizeof(float) * pcs->ldl,
                                              sizeof(float) * N, pcs->rank, cudaMemcpyHostToDevice, st));
                    Ld = p.sL;
                }
                PcSpec spec = *pcs;
                if (p.stage_l) spec.ldl = N;
                rc = build_precond(p, *kern, spec, Ld, st, &pcst, &launches, lrs ? lrs->Ct : nullptr,
                                   lrs ? lrs->rank : 0);
                if (rc != CIQ_OK) goto done;
                pc_on = true;
            }
        }
        KrylovState<R> s = krylov_state(p, op, o, tol);
        CIQ_TRY(launch_init_rhs(s, Bd, st));
        CIQ_TRY(launch_init_state(s, st));
        launches += 3 + (p.tc ? 2 : 0);
        if (prof.on) CIQ_TRY(cudaEventRecord(prof.t_pre0, st));
        if (given_nodes) {
            double hn[kNodeCount] = {0};
            double sw = 0.0;
            for (int q = 0; q < Q; ++q) { hn[kNodeW + q] = hw[q]; hn[kNodeT + q] = ht[q]; sw += hw[q]; }
            hn[kNodeLmin] = o.lmin > 0.0 ? o.lmin : 0.0;
            hn[kNodeLmax] = o.lmax > 0.0 ? o.lmax : 0.0;
            hn[kNodeSumW] = sw;
            CIQ_TRY(cudaMemcpyAsync(p.nodes, hn, sizeof(hn), cudaMemcpyHostToDevice, st));
        } else if (given_bounds) {
            CIQ_TRY(launch_nodes_from_bounds(p.nodes, Q, o.lmin, o.lmax, st));
            launches += 1;
        } else {
            CIQ_TRY(run_prepass(p, *kern, o, Q, startd, st, pc_on ? &pcst : nullptr, lr_under_pc ? &lrst : nullptr));
            launches += 3 + p.JL * (1 + (p.tc ? 4 : 1) + (pc_on ? 6 : 0));   // tensor cores: V scale, V split,
                                                                             // product, finish
        }
        if (prof.on) CIQ_TRY(cudaEventRecord(prof.t_pre1, st));
        MvmArgs<R> a = mvm_args(p, *kern);
        a.T = T;
        a.mode = kLanczos;
        a.partials = p.partials;
        a.stop = p.all_done;
        a.plo = p.plo;
        // Kernels per MVM: one on CUDA cores; on tensor cores the V split
        // and, per column group, the product and the finish (the V scale of
        // unit columns is set by the first MVM only).
        const int mvm_launches = p.tc ? 1 + 2 * ((T + tc_group_t(T) - 1) / tc_group_t(T)) : 1;
        // Stored basis on tensor cores: the V split of MVM j + 1 finishes
        // step j's vector update (q_{j+1} from p and the published scalars).
        const bool lz = p.basis && p.tc && !pc_on;
        const bool pc_map = pc_on && !pcst.lowrank;        // the result maps back through P^{+-1/2}
        CIQ_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        CIQ_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        if (prof.on) {
            for (int sl = 0; sl < 2; ++sl) {
                prof.ev[sl].resize(2 * (size_t)o.check_every + 1);
                for (auto& e : prof.ev[sl]) CIQ_TRY(cudaEventCreate(&e));
            }
            prof.mvm_ms.assign((size_t)p.jmax + 1, 0.0);
            prof.step_ms.assign((size_t)p.jmax + 1, 0.0);
            CIQ_TRY(cudaEventRecord(prof.t_loop, st));
        }
        {
            int slot = 0;
            bool pending[2] = {false, false};
            int first_j[2] = {0, 0}, count[2] = {0, 0};
            auto harvest = [&](int sl) -> cudaError_t {
                if (!prof.on) return cudaSuccess;
                for (int k = 0; k < count[sl]; ++k) {
                    float m = 0.f, q = 0.f;
                    cudaError_t e = cudaEventElapsedTime(&m, prof.ev[sl][2 * k], prof.ev[sl][2 * k + 1]);
                    if (e != cudaSuccess) return e;
                    e = cudaEventElapsedTime(&q, prof.ev[sl][2 * k + 1], prof.ev[sl][2 * k + 2]);
                    if (e != cudaSuccess) return e;
                    prof.mvm_ms[first_j[sl] + k] = m;
                    prof.step_ms[first_j[sl] + k] = q;
                }
                return cudaSuccess;
            };
            for (int j = 1; j <= p.jmax;) {
                const int jb = std::min(j + o.check_every - 1, p.jmax);
                if (prof.on) CIQ_TRY(cudaEventRecord(prof.ev[slot][0], st));
                for (int jj = j; jj <= jb; ++jj) {
                    if (p.basis) {
                        const size_t vs = (size_t)T * p.Npad;
                        a.V = p.V + (size_t)jj * vs;
                        a.qprev = p.V + (size_t)(jj - 1) * vs;
                        a.pout = p.V + (size_t)(jj + 1) * vs;
                        a.lz_q = lz && jj > 1 ? a.qprev : nullptr;
                        a.lz_sco = lz && jj > 1 ? p.sco : nullptr;
                    } else {
                        a.V = (jj & 1) ? p.QA : p.QB;
                        a.qprev = (jj & 1) ? p.QB : p.QA;
                    }
                    a.beta = p.beta + (size_t)(jj & 1) * T;
                    if (pc_on) CIQ_TRY(precond_mvm(p, pcst, a, st, jj > 1, lr_under_pc ? &lrst : nullptr));
                    else CIQ_TRY(launch_mvm(p, a, true, st, jj > 1));
                    if (prof.on) CIQ_TRY(cudaEventRecord(prof.ev[slot][2 * (jj - j) + 1], st));
                    CIQ_TRY(launch_msminres_step(s, jj, false, st, !lz));
                    if (prof.on) CIQ_TRY(cudaEventRecord(prof.ev[slot][2 * (jj - j) + 2], st));
                    launches += (lz ? 1 : 2) + mvm_launches + (p.tc && (jj == 1 || pc_on) ? 1 : 0) +
                                (pc_on ? 6 : 0);
                }
                first_j[slot] = j;
                count[slot] = jb - j + 1;
                last_j = jb;
                CIQ_TRY(cudaMemcpyAsync(&flags[slot], p.all_done, sizeof(int), cudaMemcpyDeviceToHost, st));
                CIQ_TRY(cudaEventRecord(ev[slot], st));
                bool stop = false;
                if (pending[slot ^ 1]) {
                    CIQ_TRY(cudaEventSynchronize(ev[slot ^ 1]));
                    CIQ_TRY(harvest(slot ^ 1));
                    pending[slot ^ 1] = false;
                    stop = flags[slot ^ 1] != 0;
                }
                pending[slot] = true;
                slot ^= 1;
                j = jb + 1;
                if (stop) break;
            }
            if (prof.on) {
                CIQ_TRY(cudaEventRecord(prof.t_loop_end, st));
                CIQ_TRY(cudaStreamSynchronize(st));
                for (int sl = 0; sl < 2; ++sl)
                    if (pending[sl]) CIQ_TRY(harvest(sl));
            }
        }
        CIQ_TRY(launch_msminres_step(s, last_j + 1, true, st));
        launches += 1;
        // Preconditioned: the combine forms the estimate in the space of A,
        // then P^{-1/2} (R' b) or P^{1/2} (R b) maps it back.
        R* comb = outd;
        if constexpr (sizeof(R) == 4) {
            if (pc_map) comb = p.Apre;
        }
        if (p.basis) {
            CIQ_TRY(launch_basis_combine(s, comb, last_j, st));   // kOpSqrtMvm: the sum goes to Y
            launches += 2;
        }
        if constexpr (sizeof(R) == 4) {
            if (vjp) {
                CIQ_TRY(launch_vjp(s, p.Xp, p.dp, kern->type, kern->lengthscale, kern->outputscale, p.Xq, p.vpart,
                                   p.vgrad, st));
                launches += 3 + (Q + 3) / 4;
            }
        }
        if (op == kOpSqrtMvm) {
            if (!p.basis) CIQ_TRY(launch_combine(s, outd, st));      // folds the trailing part into Y
            MvmArgs<R> m = mvm_args(p, *kern);
            m.T = T;
            m.mode = kPlain;
            m.V = p.Y;
            m.out = outd;
            m.ldo = N;
            if constexpr (sizeof(R) == 4) {
                if (lrs) {
                    // (K - C C^T) Y: the MVM into Op, the low-rank term, then out.
                    m.out = p.Op;
                    m.ldo = p.Npad;
                    CIQ_TRY(launch_mvm(p, m, false, st));
                    CIQ_TRY(launch_lowrank_apply(lr_under_pc ? lrst : pcst, p.Y, p.Op, T, nullptr, st));
                    CIQ_TRY(cudaMemcpy2DAsync(outd, sizeof(R) * N, p.Op, sizeof(R) * p.Npad, sizeof(R) * N, T,
                                              cudaMemcpyDeviceToDevice, st));
                    launches += 3;
                } else {
                    CIQ_TRY(launch_mvm(p, m, false, st));
                }
            } else {
                CIQ_TRY(launch_mvm(p, m, false, st));
            }
            launches += p.basis ? 1 : 2;
        } else if (!p.basis) {
            CIQ_TRY(launch_combine(s, comb, st));
            launches += 1;
        }
        if constexpr (sizeof(R) == 4) {
            if (pc_map) {
                if (pc_literal) {
                    // R' b into the MVM's input buffer, then R b = K (R' b).
                    CIQ_TRY(launch_pc_apply(pcst, p.Apre, N, T, true, p.Up, p.Npad, nullptr, st));
                    MvmArgs<R> m = mvm_args(p, *kern);
                    m.T = T;
                    m.mode = kPlain;
                    m.V = p.Up;
                    m.out = outd;
                    m.ldo = N;
                    if (lr_under_pc) {
                        // (K - C C^T)(R' b) for the posterior covariance.
                        m.out = p.Op;
                        m.ldo = p.Npad;
                        CIQ_TRY(launch_mvm(p, m, false, st));
                        CIQ_TRY(launch_lowrank_apply(lrst, p.Up, p.Op, T, nullptr, st));
                        CIQ_TRY(cudaMemcpy2DAsync(outd, sizeof(R) * N, p.Op, sizeof(R) * p.Npad, sizeof(R) * N, T,
                                                  cudaMemcpyDeviceToDevice, st));
                        launches += 3;
                    } else {
                        CIQ_TRY(launch_mvm(p, m, false, st));
                    }
                    launches += mvm_launches + 1;
                } else {
                    CIQ_TRY(launch_pc_apply(pcst, p.Apre, N, T, op == kOpInvSqrt, outd, N, nullptr, st));
                }
                launches += pcst.rank > 0 ? 3 : 1;
            }
            // The posterior mean, after the map back through P^{1/2}.
            const float* mu = lr_under_pc ? lrst.mu : (pc_on && pcst.lowrank ? pcst.mu : nullptr);
            if (mu) {
                CIQ_TRY(launch_add_mean(outd, N, N, T, mu, st));
                launches += 1;
            }
        }
        CIQ_TRY(launch_summary(s, last_j, st));
        launches += 1;
        if (prof.on) CIQ_TRY(cudaEventRecord(prof.t_end, st));
        if (p.stage_out)
            CIQ_TRY(cudaMemcpyAsync(out, p.sout, sizeof(R) * (size_t)N * T, cudaMemcpyDeviceToHost, st));
        CIQ_TRY(cudaMemcpyAsync(summary, p.summary, sizeof(summary), cudaMemcpyDeviceToHost, st));
        CIQ_TRY(cudaMemcpyAsync(nodes, p.nodes, sizeof(nodes), cudaMemcpyDeviceToHost, st));
        if (p.tc) CIQ_TRY(cudaMemcpyAsync(&tc_timeout, p.tcp.err, sizeof(int), cudaMemcpyDeviceToHost, st));
        if (vjp) CIQ_TRY(cudaMemcpyAsync(vjp_grad, p.vgrad, 3 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CIQ_TRY(cudaStreamSynchronize(st));
    }
done:
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    double t_total = 0, t_pre = 0, t_mvm = 0, t_step = 0;
    int n_mvm = 0, n_step = 0;
    if (prof.on && rc == CIQ_OK) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, prof.t_start, prof.t_end) == cudaSuccess) t_total = ms;
        if (cudaEventElapsedTime(&ms, prof.t_pre0, prof.t_pre1) == cudaSuccess) t_pre = ms;
        const int itmax = (int)summary[0];
        // Launches after the last working iteration return at once (every
        // column had stopped); count the one MVM that ran before the freeze.
        const int upto = std::min(itmax + 1, last_j);
        for (int jj = 1; jj <= upto; ++jj) {
            t_mvm += prof.mvm_ms[jj];
            ++n_mvm;
            if (jj <= itmax) { t_step += prof.step_ms[jj]; ++n_step; }
        }
    }
    prof.destroy();
    if (owned) {
        cudaFreeAsync(base, st);
        if (rc != CIQ_OK) cudaStreamSynchronize(st);
    }
    if (rc != CIQ_OK) {
        cudaGetLastError();
        return rc;
    }
    if (info) {
        memset(info, 0, sizeof(*info));
        info->iters = (int)summary[0];
        info->iters_min = (int)summary[1];
        info->converged = (int)summary[2];
        info->resid_max = summary[3];
        info->errbound_max = summary[4];
        info->lanczos_iters = (int)nodes[kNodeLanczosSteps];
        info->ritz_min = nodes[kNodeRitzMin];
        info->ritz_max = nodes[kNodeRitzMax];
        info->lmin_used = nodes[kNodeLmin];
        info->lmax_used = nodes[kNodeLmax];
        info->q = Q;
        for (int q = 0; q < Q; ++q) { info->w[q] = nodes[kNodeW + q]; info->t[q] = nodes[kNodeT + q]; }
        info->launches = launches;
        info->t_total_ms = t_total;
        info->t_prepass_ms = t_pre;
        info->t_mvm_ms = t_mvm;
        info->t_step_ms = t_step;
        info->mvm_launches = n_mvm;
        info->step_launches = n_step;
        info->krylov = p.basis ? CIQ_KRYLOV_BASIS : CIQ_KRYLOV_RECURRENCE;
        info->precond_rank = pc_on && !pcst.lowrank ? pcst.rank : 0;
    }
    if (tc_timeout) return CIQ_ERR_TIMEOUT;
    if (summary[6] > 0) return CIQ_ERR_NAN;
    if ((int)summary[5] == kColMaxIter) return CIQ_NOT_CONVERGED;
    return CIQ_OK;
}

// ---------------------------------------------------------------- batched --
// Host image of one work list (see DevList): problems and their first items.
struct HostList {
    std::vector<int> ids, prefix{0};
    void add(int p, int64_t items) {
        ids.push_back(p);
        prefix.push_back((int)(prefix.back() + items));
    }
    int total() const { return prefix.back(); }
};

// Stream used only to record batched iteration graphs, one per host thread
// and device (a stream belongs to the device current at its creation).
cudaStream_t capture_stream() {
    constexpr int kMaxDev = 64;
    thread_local cudaStream_t cs[kMaxDev] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) {
        cudaGetLastError();
        return nullptr;
    }
    if (!cs[dev] && cudaStreamCreateWithFlags(&cs[dev], cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cs[dev] = nullptr;
    }
    return cs[dev];
}

// Pinned host words for the list totals (two slots), one set per host thread.
int* pinned_totals() {
    thread_local int* p = nullptr;
    if (!p) {
        if (cudaHostAlloc(reinterpret_cast<void**>(&p), 2 * kBatchDynLists * sizeof(int), cudaHostAllocDefault) !=
            cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
        }
    }
    return p;
}

// record_tri: keep column 0's msMINRES tridiagonal and report its largest
// Ritz value; packed_out (optional) receives the packed per-problem results.
ciq_status solve_batched(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                         ciq_info* infos, cudaStream_t st, int op, bool record_tri = false,
                         std::vector<double>* packed_out = nullptr) {
    if (!probs || P < 1 || P > CIQ_MAX_BATCH || Q < 1 || Q > CIQ_MAX_Q || !(tol >= 0.0)) return CIQ_ERR_ARG;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    if (!valid_options(o)) return CIQ_ERR_ARG;
    if (o.mvm == CIQ_MVM_STORED || o.quad_w || o.quad_t || o.lanczos_start || o.workspace ||
        o.sqrt_form != CIQ_SQRT_IDENTITY || o.precision == CIQ_PREC_TF32)
        return CIQ_ERR_UNSUPPORTED;
    const int T = probs[0].T;
    if (T < 1) return CIQ_ERR_ARG;
    // Tensor-core batches: FP16/BF16 split tiles, one launch group (T <= 64).
    const bool tc = o.precision != CIQ_PREC_FP32;
    const bool half = o.precision == CIQ_PREC_FP16;
    if (tc && (tc_padded_t(T) < 0 || T > 64)) return CIQ_ERR_UNSUPPORTED;
    const int TP = tc ? tc_padded_t(T) : 0;
    std::vector<char> given(P);
    for (int p = 0; p < P; ++p) {
        const ciq_problem& q = probs[p];
        if (!q.X || !q.B || !q.out || q.N < 1 || q.d < 1 || q.d > CIQ_MAX_DIM || q.T != T || !valid_kernel(&q.kern))
            return CIQ_ERR_ARG;
        given[p] = q.lmin > 0.0 && q.lmax > 0.0;
        if (given[p] && !(q.lmax >= q.lmin && std::isfinite(q.lmax))) return CIQ_ERR_ARG;
        if (tc && !tc_supported(o.precision, q.d)) return CIQ_ERR_UNSUPPORTED;
        if (!device_accessible(q.X) || !device_accessible(q.B) || !device_accessible(q.out)) return CIQ_ERR_ARG;
    }
    keep_pool_warm();
    int* tot_h = pinned_totals();
    if (!tot_h) return CIQ_ERR_CUDA;

    // Per-problem workspaces (the single-problem layout), then the shared tables.
    std::vector<Plan<float>> plans;
    plans.reserve(P);
    std::vector<size_t> offs(P);
    size_t off = 0;
    for (int p = 0; p < P; ++p) {
        plans.push_back(make_plan<float>(probs[p].N, probs[p].d, T, Q, o, !given[p], tc));
        // Many problems fill the GPU; splitting a row tile's columns across
        // CTAs only adds per-CTA cost here (measured 3.78 -> 2.94 s on the
        // 512-problem batch without it), so batches default to one CTA.
        plans.back().tc_max_split = o.tc_split > 0 ? o.tc_split : 1;
        // A tuned policy: large problems (the ones left in a batch's tail, when
        // few row tiles are live) split their row tiles over more CTAs.
        if (o.batch_split_rows > 0 && plans.back().Npad / kTcBM >= o.batch_split_rows)
            plans.back().tc_max_split = o.batch_split;
        plans.back().tri_on = record_tri;
        plans.back().pair_p = true;
        plans.back().layout(nullptr);
        offs[p] = off;
        off += round_up((int64_t)plans.back().bytes, kAlign);
    }
    const int groups = (T + batch_mvm_group(T) - 1) / batch_mvm_group(T);
    std::vector<BatchProblem> hp(P);
    // Tensor-core pre-pass: MVM items per kernel type, V split and finish.
    HostList pre_tc, pre_tc_split, pre_tc_fin;
    HostList prep, one, init, pre, pre_one, given_one, fin, comb, rows256, pre_mvm[kBatchClasses],
        dyn[kBatchDynLists];
    int64_t biggest = 0;
    for (int p = 0; p < P; ++p) {
        const Plan<float>& pl = plans[p];
        BatchProblem& b = hp[p];
        b.mvm_tiles = (int)batch_mvm_row_tiles(pl.Npad, T);
        b.mvm_items = b.mvm_tiles * groups;
        b.pre_tiles = (int)(pl.Npad / 32);
        b.cls = probs[p].kern.type * 4 + pl.dp / 4 - 1;
        b.d = pl.d;
        const int64_t prep_items = (pl.Npad * pl.dp + 255) / 256;
        const int64_t comb_items = (pl.N + 255) / 256 * T;
        biggest = std::max<int64_t>({biggest, prep_items, comb_items, (int64_t)b.mvm_items,
                                     (int64_t)pl.nchunks * T});
        prep.add(p, prep_items);
        one.add(p, 1);
        rows256.add(p, (pl.Npad + 255) / 256);
        init.add(p, (int64_t)pl.nchunks * T);
        fin.add(p, T);
        comb.add(p, comb_items);
        for (int l = 0; l < kBatchDynLists; ++l) b.list_items[l] = 0;
        if (tc) {
            b.list_items[0] = (int)(pl.Npad / kTcBM) * pl.tcp.nsplit;     // both kernel types in one list
            b.list_items[kListTcSplit] = (int)((pl.Npad / 8 * TP + 255) / 256);
            b.list_items[kListTcFinish] = (int)(pl.Npad / kTcBM) * (TP / 16);   // row tile x 16 columns
        } else {
            b.list_items[b.cls] = b.mvm_items;
        }
        b.list_items[kBatchClasses] = pl.nchunks * T;
        b.list_items[kListStepScalar] = T;
        if (given[p]) {
            given_one.add(p, 1);
        } else {
            pre.add(p, pl.nchunks1);
            pre_one.add(p, 1);
            if (tc) {
                pre_tc.add(p, (int64_t)(pl.Npad / kTcBM) * pl.tcp.nsplit);
                pre_tc_split.add(p, (pl.Npad / 8 * 32 + 255) / 256);
                pre_tc_fin.add(p, (pl.Npad / kTcBM) * (32 / 16));
            } else {
                pre_mvm[b.cls].add(p, b.pre_tiles);
            }
        }
    }
    // The main-loop lists hold the problems longest first (decreasing padded
    // N: a CTA of the tensor-core MVM walks Npad / 128 column steps), so the
    // longest CTAs start in the first wave and short ones fill in behind them
    // (longest-processing-time order); the list rebuilds keep that order.
    // Each problem's arithmetic does not depend on it.
    std::vector<int> order(P);
    for (int p = 0; p < P; ++p) order[p] = p;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return plans[a].Npad > plans[b].Npad; });
    for (int q = 0; q < P; ++q) {
        const int p = order[q];
        for (int l = 0; l < kBatchDynLists; ++l)
            if (hp[p].list_items[l] > 0) dyn[l].add(p, hp[p].list_items[l]);
    }
    // Item totals index blocks as int.
    {
        int64_t sums[7] = {0, 0, 0, 0, 0, 0, 0};
        for (int p = 0; p < P; ++p) {
            const Plan<float>& pl = plans[p];
            sums[0] += (pl.Npad * pl.dp + 255) / 256;
            sums[1] += (pl.N + 255) / 256 * T;
            sums[2] += (int64_t)hp[p].mvm_items;
            sums[3] += (int64_t)pl.nchunks * T;
            sums[4] += hp[p].pre_tiles;
            sums[5] += pl.nchunks1;
            sums[6] += (pl.Npad / kTcBM) * std::max(pl.tcp.nsplit, 2);
        }
        for (int64_t v : sums)
            if (v >= (int64_t)INT32_MAX) return CIQ_ERR_UNSUPPORTED;
    }
    (void)biggest;
    std::vector<HostList*> all_lists = {&prep, &one, &init, &pre, &pre_one, &given_one, &fin, &comb, &rows256};
    for (auto& l : pre_mvm) all_lists.push_back(&l);
    all_lists.push_back(&pre_tc);
    all_lists.push_back(&pre_tc_split);
    all_lists.push_back(&pre_tc_fin);
    for (auto& l : dyn) all_lists.push_back(&l);
    const size_t list_ints = (size_t)2 * P + 2;
    const size_t tables = round_up((int64_t)(sizeof(BatchProblem) * P), kAlign) +
                          round_up((int64_t)(sizeof(int) * list_ints * all_lists.size()), kAlign) +
                          round_up((int64_t)(sizeof(int) * kBatchDynLists), kAlign) +
                          round_up((int64_t)(sizeof(int) * P), kAlign) +
                          round_up((int64_t)(sizeof(double) * kSummaryStride * P), kAlign);
    char* base = nullptr;
    ciq_status rc = CIQ_OK;
    int launches = 0;
    int last_j = 0;
    std::vector<double> packed((size_t)kSummaryStride * P, 0.0);
    std::vector<int> list_img(list_ints * all_lists.size(), 0);
    cudaEvent_t ev[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec = nullptr;
    bool capturing = false;
    {
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), off + tables, st);
        if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    }
    {
        char* tb = base + off;
        BatchProblem* probs_d = reinterpret_cast<BatchProblem*>(tb);
        tb += round_up((int64_t)(sizeof(BatchProblem) * P), kAlign);
        int* lists_d = reinterpret_cast<int*>(tb);
        tb += round_up((int64_t)(sizeof(int) * list_ints * all_lists.size()), kAlign);
        int* totals_d = reinterpret_cast<int*>(tb);
        tb += round_up((int64_t)(sizeof(int) * kBatchDynLists), kAlign);
        int* order_d = reinterpret_cast<int*>(tb);
        tb += round_up((int64_t)(sizeof(int) * P), kAlign);
        double* packed_d = reinterpret_cast<double*>(tb);
        // Device lists: [np][ids P][prefix P + 1] each.
        std::vector<DevList> dl(all_lists.size());
        for (size_t l = 0; l < all_lists.size(); ++l) {
            int* img = list_img.data() + l * list_ints;
            const HostList& h = *all_lists[l];
            img[0] = (int)h.ids.size();
            std::copy(h.ids.begin(), h.ids.end(), img + 1);
            std::copy(h.prefix.begin(), h.prefix.end(), img + 1 + P);
            int* d = lists_d + l * list_ints;
            dl[l] = DevList{d, d + 1, d + 1 + P};
        }
        auto L = [&](const HostList& h) {
            for (size_t l = 0; l < all_lists.size(); ++l)
                if (all_lists[l] == &h) return dl[l];
            return DevList{};
        };
        DynLists dyn_d;
        for (int l = 0; l < kBatchDynLists; ++l) dyn_d.l[l] = L(dyn[l]);
        for (int p = 0; p < P; ++p) {
            Plan<float>& pl = plans[p];
            pl.layout(base + offs[p]);
            BatchProblem& b = hp[p];
            const ciq_kernel& k = probs[p].kern;
            b.ks = krylov_state(pl, op, o, tol);
            b.ls = lanczos_state(pl);
            MvmArgs<float> a = mvm_args(pl, k);
            for (int par = 0; par < 2; ++par) {
                MvmArgs<float> m = a;
                m.T = T;
                m.mode = kLanczos;
                m.partials = pl.partials;
                m.stop = pl.all_done;
                m.V = par ? pl.QA : pl.QB;
                m.qprev = par ? pl.QB : pl.QA;
                m.beta = pl.beta + (size_t)par * T;
                m.plo = pl.plo;
                b.mvm[par] = m;
                MvmArgs<float> r = a;
                r.T = 1;
                r.mode = kLanczos;
                r.partials = pl.lpart;
                r.stop = pl.ldone;
                r.V = par ? pl.LA : pl.LB;
                r.qprev = par ? pl.LB : pl.LA;
                r.beta = pl.bpar ? pl.bpar + par : nullptr;
                b.pre[par] = r;
            }
            b.tcp = pl.tcp;
            b.X = probs[p].X;
            b.B = probs[p].B;
            b.out = probs[p].out;
            b.Xp = pl.Xp;
            b.nodes = pl.nodes;
            b.inv_ls = 1.0 / k.lengthscale;
            b.noise = k.noise;
            b.lmin = probs[p].lmin;
            b.lmax = probs[p].lmax;
        }
        CIQ_TRY(cudaMemcpyAsync(probs_d, hp.data(), sizeof(BatchProblem) * P, cudaMemcpyHostToDevice, st));
        CIQ_TRY(cudaMemcpyAsync(lists_d, list_img.data(), sizeof(int) * list_img.size(), cudaMemcpyHostToDevice, st));
        CIQ_TRY(cudaMemcpyAsync(order_d, order.data(), sizeof(int) * P, cudaMemcpyHostToDevice, st));
        auto setup = [&](int phase, const HostList& h) -> cudaError_t {
            if (h.total() == 0) return cudaSuccess;
            ++launches;
            return launch_batched_setup(probs_d, phase, o.seed, Q, L(h), h.total(), st);
        };
        CIQ_TRY(setup(kBatchPrepare, prep));
        if (tc) {
            CIQ_TRY(launch_batched_tc_mean(probs_d, L(one), one.total(), st));
            CIQ_TRY(launch_batched_tc_points(probs_d, L(rows256), rows256.total(), half, st));
            launches += 2;
        }
        CIQ_TRY(setup(kBatchReset, one));
        CIQ_TRY(setup(kBatchInitRhs, init));
        CIQ_TRY(setup(kBatchInitState, init));
        CIQ_TRY(setup(kBatchNodesGiven, given_one));
        if (pre.total() > 0) {
            CIQ_TRY(setup(kBatchPreInitA, pre));
            CIQ_TRY(setup(kBatchPreInitB, pre));
            // Tensor-core batches run the pre-pass MVM on tensor cores too, as
            // a single solve does (one column in a 32-column group).
            if (tc) CIQ_TRY(prepare_batched_tc_mvm(32, half));
            for (int j = 1; j <= o.lanczos_iters; ++j) {
                if (tc) {
                    CIQ_TRY(launch_batched_tc_split(probs_d, j & 1, L(pre_tc_split), pre_tc_split.total(), half, true,
                                                    st));
                    CIQ_TRY(launch_batched_tc_mvm(probs_d, 32, half, j & 1, true, L(pre_tc), pre_tc.total(), st));
                    CIQ_TRY(launch_batched_tc_finish(probs_d, 32, j & 1, true, L(pre_tc_fin), pre_tc_fin.total(), st));
                    launches += 3;
                }
                for (int c = 0; c < kBatchClasses; ++c) {
                    if (pre_mvm[c].total() == 0) continue;
                    CIQ_TRY(launch_batched_mvm(probs_d, c, T, true, j & 1, L(pre_mvm[c]), pre_mvm[c].total(), st));
                    ++launches;
                }
                CIQ_TRY(launch_batched_lanczos_step(probs_d, j, L(pre), pre.total(), st));
                ++launches;
            }
            CIQ_TRY(launch_batched_bounds_nodes(probs_d, Q, o.lmax_margin, o.lmin_div, L(pre_one), pre_one.total(), st));
            ++launches;
        }
        int grid[kBatchDynLists];
        for (int l = 0; l < kBatchDynLists; ++l) grid[l] = dyn[l].total();
        CIQ_TRY(cudaEventCreateWithFlags(&ev[0], cudaEventDisableTiming));
        CIQ_TRY(cudaEventCreateWithFlags(&ev[1], cudaEventDisableTiming));
        {
            int slot = 0;
            bool pending[2] = {false, false};
            if (tc) CIQ_TRY(prepare_batched_tc_mvm(TP, half));   // kernel attributes, outside any capture
            for (int j = 1; j <= o.max_iter;) {
                const int jb = std::min(j + o.check_every - 1, o.max_iter);
                // One batch of iterations (and the list rebuild): captured as a
                // graph and launched as one when o.graph, else launched directly.
                // The graph keeps its instantiation while only kernel
                // parameters and grid sizes change between batches.
                // Captured on a private stream (capture is not allowed on the
                // legacy default stream); the graph is launched on `st`.
                cudaStream_t ls = st;
                if (o.graph) {
                    ls = capture_stream();
                    if (!ls) { rc = CIQ_ERR_CUDA; goto done; }
                    CIQ_TRY(cudaStreamBeginCapture(ls, cudaStreamCaptureModeThreadLocal));
                    capturing = true;
                }
                for (int jj = j; jj <= jb; ++jj) {
                    if (tc) {
                        if (grid[kListTcSplit] > 0) {
                            CIQ_TRY(launch_batched_tc_split(probs_d, jj & 1, dyn_d.l[kListTcSplit], grid[kListTcSplit],
                                                            half, false, ls));
                            ++launches;
                        }
                        if (grid[0] > 0) {
                            CIQ_TRY(launch_batched_tc_mvm(probs_d, TP, half, jj & 1, false, dyn_d.l[0], grid[0], ls));
                            ++launches;
                        }
                        if (grid[kListTcFinish] > 0) {
                            CIQ_TRY(launch_batched_tc_finish(probs_d, TP, jj & 1, false, dyn_d.l[kListTcFinish],
                                                             grid[kListTcFinish], ls));
                            ++launches;
                        }
                    } else {
                        for (int c = 0; c < kBatchClasses; ++c) {
                            if (grid[c] == 0) continue;
                            CIQ_TRY(launch_batched_mvm(probs_d, c, T, false, jj & 1, dyn_d.l[c], grid[c], ls));
                            ++launches;
                        }
                    }
                    CIQ_TRY(launch_batched_step_scalar(probs_d, jj, false, dyn_d.l[kListStepScalar],
                                                       grid[kListStepScalar], ls));
                    CIQ_TRY(launch_batched_step_vector(probs_d, jj, dyn_d.l[kBatchClasses], grid[kBatchClasses], ls));
                    launches += 2;
                }
                last_j = jb;
                CIQ_TRY(launch_rebuild_lists(probs_d, P, order_d, dyn_d, totals_d, ls));
                ++launches;
                if (o.graph) {
                    cudaGraph_t g = nullptr;
                    capturing = false;
                    CIQ_TRY(cudaStreamEndCapture(ls, &g));
                    if (gexec) {
                        cudaGraphExecUpdateResultInfo ui;
                        if (cudaGraphExecUpdate(gexec, g, &ui) != cudaSuccess) {
                            cudaGetLastError();
                            cudaGraphExecDestroy(gexec);
                            gexec = nullptr;
                        }
                    }
                    cudaError_t ge = gexec ? cudaSuccess : cudaGraphInstantiate(&gexec, g, 0);
                    cudaGraphDestroy(g);
                    CIQ_TRY(ge);
                    CIQ_TRY(cudaGraphLaunch(gexec, st));
                }
                CIQ_TRY(cudaMemcpyAsync(tot_h + slot * kBatchDynLists, totals_d, sizeof(int) * kBatchDynLists,
                                        cudaMemcpyDeviceToHost, st));
                CIQ_TRY(cudaEventRecord(ev[slot], st));
                bool stop = false;
                if (pending[slot ^ 1]) {
                    CIQ_TRY(cudaEventSynchronize(ev[slot ^ 1]));
                    pending[slot ^ 1] = false;
                    // Totals of the previous rebuild bound the lists the next
                    // launches read (lists only shrink).
                    for (int l = 0; l < kBatchDynLists; ++l) grid[l] = tot_h[(slot ^ 1) * kBatchDynLists + l];
                    stop = grid[kBatchClasses] == 0;
                }
                pending[slot] = true;
                slot ^= 1;
                j = jb + 1;
                if (stop) break;
            }
        }
        CIQ_TRY(launch_batched_step_scalar(probs_d, last_j + 1, true, L(fin), fin.total(), st));
        CIQ_TRY(setup(kBatchCombine, comb));
        CIQ_TRY(launch_batched_summary(probs_d, last_j, packed_d, L(one), one.total(), st));
        launches += 2;
        CIQ_TRY(cudaMemcpyAsync(packed.data(), packed_d, sizeof(double) * packed.size(), cudaMemcpyDeviceToHost, st));
        CIQ_TRY(cudaStreamSynchronize(st));
    }
done:
    if (capturing) {
        cudaGraph_t g = nullptr;
        cudaStreamEndCapture(capture_stream(), &g);
        if (g) cudaGraphDestroy(g);
        cudaGetLastError();
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (ev[0]) cudaEventDestroy(ev[0]);
    if (ev[1]) cudaEventDestroy(ev[1]);
    cudaFreeAsync(base, st);
    if (rc != CIQ_OK) {
        cudaStreamSynchronize(st);
        cudaGetLastError();
        return rc;
    }
    bool any_nan = false, any_maxit = false, any_timeout = false;
    for (int p = 0; p < P; ++p) {
        const double* sm = packed.data() + (size_t)p * kSummaryStride;
        const double* nd = sm + 8;
        if (sm[9 + kNodeCount] != 0.0) any_timeout = true;
        if (sm[6] > 0) any_nan = true;
        if ((int)sm[5] == kColMaxIter) any_maxit = true;
        if (!infos) continue;
        ciq_info* info = infos + p;
        memset(info, 0, sizeof(*info));
        info->iters = (int)sm[0];
        info->iters_min = (int)sm[1];
        info->converged = (int)sm[2];
        info->resid_max = sm[3];
        info->errbound_max = sm[4];
        info->lanczos_iters = (int)nd[kNodeLanczosSteps];
        info->ritz_min = nd[kNodeRitzMin];
        info->ritz_max = nd[kNodeRitzMax];
        info->lmin_used = nd[kNodeLmin];
        info->lmax_used = nd[kNodeLmax];
        info->q = Q;
        for (int q = 0; q < Q; ++q) { info->w[q] = nd[kNodeW + q]; info->t[q] = nd[kNodeT + q]; }
        info->launches = launches;
        info->ritz_max_solve = sm[8 + kNodeCount];
    }
    if (packed_out) packed_out->swap(packed);
    if (any_timeout) return CIQ_ERR_TIMEOUT;
    if (any_nan) return CIQ_ERR_NAN;
    if (any_maxit) return CIQ_NOT_CONVERGED;
    return CIQ_OK;
}

// Batched solve with bounds predicted by the network; fallback to the
// Lanczos pre-pass for problems whose own Krylov space contradicts them.
ciq_status solve_batched_learned(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                                 const float* theta, double margin, ciq_info* infos, int* fallback,
                                 cudaStream_t st, int op) {
    if (!probs || P < 1 || P > CIQ_MAX_BATCH || !theta || !std::isfinite(margin)) return CIQ_ERR_ARG;
    if (!device_accessible(theta)) return CIQ_ERR_ARG;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    if (!valid_options(o)) return CIQ_ERR_ARG;
    for (int p = 0; p < P; ++p)
        if (!probs[p].X || probs[p].N < 1 || probs[p].d < 1 || probs[p].d > CIQ_MAX_DIM ||
            !valid_kernel(&probs[p].kern) || !device_accessible(probs[p].X))
            return CIQ_ERR_ARG;
    keep_pool_warm();
    std::vector<float> pred((size_t)P * kMlpOut);
    {
        char* base = nullptr;
        const size_t b0 = round_up((int64_t)(sizeof(ciq_problem) * P), kAlign);
        const size_t b1 = round_up((int64_t)(sizeof(float) * P * kMlpIn), kAlign);
        cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), b0 + b1 + sizeof(float) * P * kMlpOut, st);
        if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
        ciq_problem* pd = reinterpret_cast<ciq_problem*>(base);
        float* F = reinterpret_cast<float*>(base + b0);
        float* Yp = reinterpret_cast<float*>(base + b0 + b1);
        e = cudaMemcpyAsync(pd, probs, sizeof(ciq_problem) * P, cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess) e = launch_mlp_features(pd, P, F, st);
        if (e == cudaSuccess) e = launch_mlp_predict(theta, F, P, Yp, 1, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(pred.data(), Yp, sizeof(float) * pred.size(), cudaMemcpyDeviceToHost, st);
        cudaFreeAsync(base, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) { cudaStreamSynchronize(st); cudaGetLastError(); return from_cuda(e); }
    }
    std::vector<ciq_problem> mod(probs, probs + P);
    std::vector<char> predicted(P, 0);
    for (int p = 0; p < P; ++p) {
        if (mod[p].lmin > 0.0 && mod[p].lmax > 0.0) continue;
        const double noise = mod[p].kern.noise;
        const double lmax = o.lmax_margin * std::exp((double)pred[(size_t)p * kMlpOut + 1] + margin);
        const double lmin = noise > 0.0 ? noise : std::exp((double)pred[(size_t)p * kMlpOut]) / o.lmin_div;
        if (!(lmin > 0.0) || !std::isfinite(lmax)) continue;       // leave this one to the pre-pass
        mod[p].lmin = lmin;
        mod[p].lmax = std::max(lmax, lmin);
        predicted[p] = 1;
    }
    std::vector<ciq_info> own;
    if (!infos) {
        own.resize(P);
        infos = own.data();
    }
    std::vector<double> packed;
    ciq_status rc = solve_batched(mod.data(), P, Q, tol, &o, infos, st, op, true, &packed);
    if (rc != CIQ_OK && rc != CIQ_NOT_CONVERGED && rc != CIQ_ERR_NAN) return rc;
    std::vector<int> redo;
    for (int p = 0; p < P; ++p) {
        const double* sm = packed.data() + (size_t)p * kSummaryStride;
        const bool nan = sm[6] > 0;
        const bool above = sm[8 + kNodeCount] > sm[8 + kNodeLmax] * (1.0 + 1e-6);
        const bool bad = predicted[p] && (nan || above);
        if (fallback) fallback[p] = bad ? 1 : 0;
        if (bad) redo.push_back(p);
    }
    std::vector<char> nan_p(P), maxit_p(P);
    for (int p = 0; p < P; ++p) {
        const double* sm = packed.data() + (size_t)p * kSummaryStride;
        nan_p[p] = sm[6] > 0;
        maxit_p[p] = (int)sm[5] == kColMaxIter;
    }
    if (!redo.empty()) {
        std::vector<ciq_problem> sub;
        for (int p : redo) {
            ciq_problem q = probs[p];
            q.lmin = q.lmax = 0.0;
            sub.push_back(q);
        }
        std::vector<ciq_info> sub_infos(redo.size());
        std::vector<double> packed2;
        const ciq_status rc2 = solve_batched(sub.data(), (int)sub.size(), Q, tol, &o, sub_infos.data(), st, op, true,
                                             &packed2);
        if (rc2 != CIQ_OK && rc2 != CIQ_NOT_CONVERGED && rc2 != CIQ_ERR_NAN) return rc2;
        for (size_t k = 0; k < redo.size(); ++k) {
            const int p = redo[k];
            infos[p] = sub_infos[k];
            const double* sm = packed2.data() + k * kSummaryStride;
            nan_p[p] = sm[6] > 0;
            maxit_p[p] = (int)sm[5] == kColMaxIter;
        }
    }
    for (int p = 0; p < P; ++p)
        if (nan_p[p]) return CIQ_ERR_NAN;
    for (int p = 0; p < P; ++p)
        if (maxit_p[p]) return CIQ_NOT_CONVERGED;
    return CIQ_OK;
}

}  // namespace

// ------------------------------------------------------------ C entry points --
extern "C" {

const char* ciq_status_string(int status) {
    switch (status) {
        case CIQ_OK: return "ok";
        case CIQ_ERR_ARG: return "invalid argument";
        case CIQ_ERR_CUDA: return "CUDA error";
        case CIQ_ERR_NOMEM: return "out of device memory";
        case CIQ_NOT_CONVERGED: return "not converged within max_iter";
        case CIQ_ERR_NAN: return "non-finite Lanczos coefficient";
        case CIQ_ERR_UNSUPPORTED: return "unsupported option";
        case CIQ_ERR_SCRATCH_TOO_SMALL: return "problem exceeds the static scratch of the allocation-free entry point";
        case CIQ_ERR_TIMEOUT: return "a bounded wait of the tensor-core MVM gave up";
        default: return "unknown status";
    }
}

void ciq_default_options(ciq_options* opt) {
    if (!opt) return;
    memset(opt, 0, sizeof(*opt));
    opt->precision = CIQ_PREC_FP32;
    opt->mvm = CIQ_MVM_AUTO;
    opt->stop_rule = CIQ_STOP_RESIDUAL;
    opt->sqrt_form = CIQ_SQRT_IDENTITY;
    opt->max_iter = 200;
    opt->lanczos_iters = 10;
    opt->check_every = 8;
    opt->seed = 0x5eed;
    opt->lmax_margin = 1.05;
    opt->lmin_div = 100.0;
    opt->graph = 1;
}

ciq_status ciq_quad_nodes(double lmin, double lmax, int Q, double* w, double* t) {
    if (!w || !t || !(lmin > 0.0) || !(lmax >= lmin) || !std::isfinite(lmax) || Q < 1 || Q > CIQ_MAX_Q)
        return CIQ_ERR_ARG;
    return quad_nodes(lmin, lmax, Q, w, t) == 0 ? CIQ_OK : CIQ_ERR_ARG;
}

ciq_status ciq_sqrt(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, int T,
                    int Q, double tol, const ciq_options* opt, float* out, ciq_info* info,
                    ciq_stream_t stream) {
    return solve<float>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream,
                        kOpSqrtIdentity, false);
}

// Backward pass: one solve over [B | G] (2T columns), then the contractions.
static ciq_status solve_vjp(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, const float* G,
                     int T, int Q, double tol, const ciq_options* opt, float* out, float* grad_B, double* grad_theta,
                     ciq_info* info, cudaStream_t st, int op) {
    if (!X || !B || !G || !out || !grad_B || !grad_theta || N < 1 || T < 1 || T > (1 << 20)) return CIQ_ERR_ARG;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    if (!valid_options(o)) return CIQ_ERR_ARG;
    if (o.krylov == CIQ_KRYLOV_RECURRENCE || o.sqrt_form == CIQ_SQRT_MVM) return CIQ_ERR_UNSUPPORTED;
    keep_pool_warm();
    const size_t cols = sizeof(float) * (size_t)N * T;
    float *BG = nullptr, *OG = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&BG), 2 * cols, st);
    if (e == cudaSuccess) e = cudaMallocAsync(reinterpret_cast<void**>(&OG), 2 * cols, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(BG, B, cols, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(BG + (size_t)N * T, G, cols, cudaMemcpyDefault, st);
    ciq_status rc = from_cuda(e);
    if (rc == CIQ_OK) {
        rc = solve<float>(X, N, d, kern, BG, 2 * T, Q, tol, &o, OG, info, st, op, false, nullptr, 0, grad_theta);
        if (rc == CIQ_OK || rc == CIQ_NOT_CONVERGED) {
            e = cudaMemcpyAsync(out, OG, cols, cudaMemcpyDefault, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(grad_B, OG + (size_t)N * T, cols, cudaMemcpyDefault, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = from_cuda(e);
        }
    }
    if (BG) cudaFreeAsync(BG, st);
    if (OG) cudaFreeAsync(OG, st);
    if (rc != CIQ_OK && rc != CIQ_NOT_CONVERGED) cudaGetLastError();
    return rc;
}

// An explicit matrix: the kernel here only carries the absent noise term.
static const ciq_kernel kDenseKernel = {CIQ_RBF, 1.0, 1.0, 0.0};

ciq_status ciq_sqrt_dense(const float* K, int64_t N, int64_t ldk, const float* B, int T, int Q, double tol,
                          const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream) {
    if (!K) return CIQ_ERR_ARG;
    return solve<float>(nullptr, N, 1, &kDenseKernel, B, T, Q, tol, opt, out, info, (cudaStream_t)stream,
                        kOpSqrtIdentity, false, K, ldk);
}

ciq_status ciq_invsqrt_dense(const float* K, int64_t N, int64_t ldk, const float* B, int T, int Q, double tol,
                             const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream) {
    if (!K) return CIQ_ERR_ARG;
    return solve<float>(nullptr, N, 1, &kDenseKernel, B, T, Q, tol, opt, out, info, (cudaStream_t)stream,
                        kOpInvSqrt, false, K, ldk);
}

ciq_status ciq_invsqrt(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, int T,
                       int Q, double tol, const ciq_options* opt, float* out, ciq_info* info,
                       ciq_stream_t stream) {
    return solve<float>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream, kOpInvSqrt,
                        false);
}

ciq_status ciq_sqrt_f64(const double* X, int64_t N, int d, const ciq_kernel* kern, const double* B,
                        int T, int Q, double tol, const ciq_options* opt, double* out, ciq_info* info,
                        ciq_stream_t stream) {
    return solve<double>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream,
                         kOpSqrtIdentity, true);
}

ciq_status ciq_invsqrt_f64(const double* X, int64_t N, int d, const ciq_kernel* kern, const double* B,
                           int T, int Q, double tol, const ciq_options* opt, double* out,
                           ciq_info* info, ciq_stream_t stream) {
    return solve<double>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream, kOpInvSqrt,
                         true);
}

ciq_status ciq_lanczos_bounds(const float* X, int64_t N, int d, const ciq_kernel* kern, int iters,
                              uint64_t seed, const float* start, double* ritz_min, double* ritz_max,
                              double* lmin_used, double* lmax_used, ciq_stream_t stream) {
    if (!X || N < 1 || d < 1 || d > CIQ_MAX_DIM || iters < 1 || iters > 512 || !valid_kernel(kern))
        return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ciq_options o;
    ciq_default_options(&o);
    o.lanczos_iters = iters;
    o.seed = seed;
    o.max_iter = 1;
    keep_pool_warm();
    Plan<float> p = make_plan<float>(N, d, 1, 1, o, true, false);
    p.stage_x = !device_accessible(X);
    p.stage_start = start && !device_accessible(start);
    p.layout(nullptr);
    char* base = nullptr;
    ciq_status rc = CIQ_OK;
    double nodes[kNodeCount] = {0};
    cudaError_t e0 = cudaMallocAsync(reinterpret_cast<void**>(&base), p.bytes, st);
    if (e0 != cudaSuccess) { cudaGetLastError(); return from_cuda(e0); }
    {
        p.layout(base);
        const float* Xd = X;
        const float* sd = start;
        if (p.stage_x) {
            CIQ_TRY(cudaMemcpyAsync(p.sx, X, sizeof(float) * (size_t)N * d, cudaMemcpyHostToDevice, st));
            Xd = p.sx;
        }
        if (p.stage_start) {
            CIQ_TRY(cudaMemcpyAsync(p.sstart, start, sizeof(float) * (size_t)N, cudaMemcpyHostToDevice, st));
            sd = p.sstart;
        }
        CIQ_TRY(launch_prepare_points<float, float>(Xd, N, d, p.Npad, p.dp, 1.0 / kern->lengthscale, p.Xp, st));
        CIQ_TRY(run_prepass(p, *kern, o, 1, sd, st));
        CIQ_TRY(cudaMemcpyAsync(nodes, p.nodes, sizeof(nodes), cudaMemcpyDeviceToHost, st));
        CIQ_TRY(cudaStreamSynchronize(st));
    }
done:
    cudaFreeAsync(base, st);
    if (rc != CIQ_OK) { cudaStreamSynchronize(st); cudaGetLastError(); return rc; }
    if (ritz_min) *ritz_min = nodes[kNodeRitzMin];
    if (ritz_max) *ritz_max = nodes[kNodeRitzMax];
    if (lmin_used) *lmin_used = nodes[kNodeLmin];
    if (lmax_used) *lmax_used = nodes[kNodeLmax];
    return CIQ_OK;
}

}  // extern "C"

namespace {
template <typename R>
ciq_status kernel_mvm_impl(const R* X, int64_t N, int d, const ciq_kernel* kern, const R* V, int T,
                           R* out, int precision, cudaStream_t st) {
    if (!X || !V || !out || N < 1 || d < 1 || d > CIQ_MAX_DIM || T < 1 || !valid_kernel(kern) ||
        precision < CIQ_PREC_FP32 || precision > CIQ_PREC_FP16)
        return CIQ_ERR_ARG;
    const bool tc = sizeof(R) == 4 && precision != CIQ_PREC_FP32;
    if (tc && (!tc_supported(precision, d) || tc_padded_t(T) < 0)) return CIQ_ERR_UNSUPPORTED;
    if (!device_accessible(X) || !device_accessible(V) || !device_accessible(out)) return CIQ_ERR_ARG;
    keep_pool_warm();
    ciq_options o;
    ciq_default_options(&o);
    o.max_iter = 1;
    o.precision = precision;
    Plan<R> p = make_plan<R>(N, d, T, 1, o, false, tc);
    char* base = nullptr;
    ciq_status rc = CIQ_OK;
    cudaError_t e0 = cudaMallocAsync(reinterpret_cast<void**>(&base), p.bytes, st);
    if (e0 != cudaSuccess) { cudaGetLastError(); return from_cuda(e0); }
    {
        p.layout(base);
        CIQ_TRY(launch_prepare_points<R, R>(X, N, d, p.Npad, p.dp, 1.0 / kern->lengthscale, p.Xp, st));
        CIQ_TRY(tc_prepare(p, kern->type, st));
        // Zero-padded copy of V (the MVM reads whole tiles).
        CIQ_TRY(cudaMemsetAsync(p.QA, 0, sizeof(R) * (size_t)T * p.Npad, st));
        CIQ_TRY(cudaMemcpy2DAsync(p.QA, sizeof(R) * p.Npad, V, sizeof(R) * N, sizeof(R) * N, T,
                                  cudaMemcpyDeviceToDevice, st));
        MvmArgs<R> a = mvm_args(p, *kern);
        a.T = T;
        a.mode = kPlain;
        a.V = p.QA;
        a.out = out;
        a.ldo = N;
        CIQ_TRY(launch_mvm(p, a, false, st));
    }
done:
    cudaFreeAsync(base, st);
    if (rc != CIQ_OK) cudaGetLastError();
    return rc;
}
}  // namespace

extern "C" {

ciq_status ciq_kernel_mvm(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* V, int T,
                          float* out, int precision, ciq_stream_t stream) {
    return kernel_mvm_impl<float>(X, N, d, kern, V, T, out, precision, (cudaStream_t)stream);
}

ciq_status ciq_kernel_mvm_f64(const double* X, int64_t N, int d, const ciq_kernel* kern, const double* V,
                              int T, double* out, ciq_stream_t stream) {
    return kernel_mvm_impl<double>(X, N, d, kern, V, T, out, CIQ_PREC_FP32, (cudaStream_t)stream);
}

ciq_status ciq_kernel_matrix(const float* X, int64_t N, int d, const ciq_kernel* kern, float* Kmat,
                             int64_t ldk, ciq_stream_t stream) {
    const int64_t Npad = round_up(N, kRowPad);
    if (!X || !Kmat || N < 1 || d < 1 || d > CIQ_MAX_DIM || !valid_kernel(kern) || ldk < Npad || ldk % 4 != 0)
        return CIQ_ERR_ARG;
    if (!device_accessible(X) || !device_accessible(Kmat)) return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    const int dp = dim_pad(d);
    float* Xp = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&Xp), sizeof(float) * (size_t)Npad * dp, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    e = launch_prepare_points<float, float>(X, N, d, Npad, dp, 1.0 / kern->lengthscale, Xp, st);
    if (e == cudaSuccess)
        e = launch_kernel_matrix(Xp, N, Npad, dp, kern->type, (float)kern->outputscale, (float)kern->noise, Kmat, ldk,
                                 Npad, st);
    cudaFreeAsync(Xp, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    return CIQ_OK;
}

ciq_status ciq_stored_mvm(const float* Kmat, int64_t N, int64_t ldk, const float* V, int T, float* out,
                          int precision, ciq_stream_t stream) {
    const int64_t Npad = round_up(N, kRowPad);
    if (!Kmat || !V || !out || N < 1 || T < 1 || ldk < Npad || ldk % 4 != 0 || precision < CIQ_PREC_FP32 ||
        precision > CIQ_PREC_FP16)
        return CIQ_ERR_ARG;
    const bool tc = precision != CIQ_PREC_FP32;
    if (tc && (precision == CIQ_PREC_TF32 || tc_padded_t(T) < 0 || (reinterpret_cast<uintptr_t>(Kmat) & 15) != 0))
        return CIQ_ERR_UNSUPPORTED;
    if (!device_accessible(Kmat) || !device_accessible(V) || !device_accessible(out)) return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    // Zero-padded copy of V, and for the tensor cores the split-operand
    // buffers and the largest diagonal entry (it sets K's power-of-two scale).
    const size_t vbytes = round_up(sizeof(float) * (size_t)T * Npad, (size_t)kAlign);
    const size_t tbytes = tc ? tc_points_bytes(Npad, T) + kAlign : 0;
    char* base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), vbytes + tbytes + kAlign, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    float* Vp = reinterpret_cast<float*>(base);
    e = cudaMemsetAsync(Vp, 0, sizeof(float) * (size_t)T * Npad, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(Vp, sizeof(float) * Npad, V, sizeof(float) * N, sizeof(float) * N, T,
                              cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) {
        MvmArgs<float> a{};
        a.N = N;
        a.Npad = Npad;
        a.V = Vp;
        a.ldv = Npad;
        a.T = T;
        a.mode = kPlain;
        a.out = out;
        a.ldo = N;
        if (!tc) {
            e = launch_stored_mvm(Kmat, ldk, a, st);
        } else {
            TcPoints tp = tc_points_layout(base + vbytes, Npad, T, precision, 8, 1);
            float* dmax = reinterpret_cast<float*>(base + vbytes + tbytes);
            float hmax = 0.f;
            e = cudaMemsetAsync(tp.err, 0, sizeof(int), st);
            if (e == cudaSuccess) e = launch_stored_diag_max(Kmat, ldk, N, dmax, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&hmax, dmax, sizeof(float), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) e = launch_stored_mvm_tc(Kmat, ldk, tp, a, stored_tc_scale(hmax), false, st);
        }
    }
    cudaFreeAsync(base, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    return CIQ_OK;
}

ciq_status ciq_sqrt_precond(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, const float* L,
                            int64_t ldl, const float* B, int T, int Q, double tol, const ciq_options* opt, float* out,
                            ciq_info* info, ciq_stream_t stream) {
    const PcSpec spec{L, ldl, rank};
    return solve<float>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream, kOpSqrtIdentity, false,
                        nullptr, 0, nullptr, &spec);
}

ciq_status ciq_invsqrt_precond(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, const float* L,
                               int64_t ldl, const float* B, int T, int Q, double tol, const ciq_options* opt,
                               float* out, ciq_info* info, ciq_stream_t stream) {
    const PcSpec spec{L, ldl, rank};
    return solve<float>(X, N, d, kern, B, T, Q, tol, opt, out, info, (cudaStream_t)stream, kOpInvSqrt, false,
                        nullptr, 0, nullptr, &spec);
}

ciq_status ciq_pivoted_cholesky(const float* X, int64_t N, int d, const ciq_kernel* kern, int rank, float* L,
                                int64_t ldl, int64_t* piv, int* rank_out, ciq_stream_t stream) {
    if (!X || !L || N < 1 || d < 1 || d > CIQ_MAX_DIM || rank < 1 || rank > kPcMaxRank || rank > N || ldl < N ||
        !valid_kernel(kern))
        return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    const int64_t Npad = round_up(N, kRowPad);
    const int dp = dim_pad(d);
    const bool stage_x = !device_accessible(X);
    Arena ar;
    auto lay = [&](char* base) {
        ar = Arena{};
        ar.base = base;
        struct { float *Xs, *Xp, *Lf; double* dres; int *piv, *rk; void* work; } b;
        b.Xs = stage_x ? ar.take<float>((size_t)N * d) : nullptr;
        b.Xp = ar.take<float>((size_t)Npad * dp);
        b.Lf = ar.take<float>((size_t)rank * Npad);
        b.dres = ar.take<double>((size_t)Npad);
        b.piv = ar.take<int>((size_t)rank + 1);
        b.rk = ar.take<int>(1);
        b.work = ar.take<char>(pc_cholesky_work_bytes(Npad));
        return b;
    };
    lay(nullptr);
    const size_t need = ar.off + kAlign;
    char* base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), need, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    auto b = lay(base);
    std::vector<int> hp((size_t)rank + 1, 0);
    int got = 0;
    const float* Xd = X;
    if (stage_x) {
        e = cudaMemcpyAsync(b.Xs, X, sizeof(float) * (size_t)N * d, cudaMemcpyHostToDevice, st);
        Xd = b.Xs;
    }
    if (e == cudaSuccess)
        e = launch_prepare_points<float, float>(Xd, N, d, Npad, dp, 1.0 / kern->lengthscale, b.Xp, st);
    if (e == cudaSuccess)
        e = launch_pivoted_cholesky(b.Xp, N, Npad, dp, kern->type, (float)kern->outputscale, rank, b.Lf, b.piv,
                                    b.dres, b.work, b.rk, st);
    if (e == cudaSuccess)
        e = cudaMemcpy2DAsync(L, sizeof(float) * ldl, b.Lf, sizeof(float) * Npad, sizeof(float) * N, rank,
                              cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hp.data(), b.piv, sizeof(int) * rank, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&got, b.rk, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess && piv) {
        std::vector<int64_t> p64(rank);
        for (int k = 0; k < rank; ++k) p64[k] = k < got ? hp[k] : -1;
        e = cudaMemcpy(piv, p64.data(), sizeof(int64_t) * rank, cudaMemcpyDefault);
    }
    cudaFreeAsync(base, st);
    cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    if (rank_out) *rank_out = got;
    return CIQ_OK;
}

ciq_status ciq_posterior_sample(const float* Xtr, int64_t n, const float* y, const float* Xc, int64_t Nc, int d,
                                int kernel_type, const double* lengthscales, double outputscale, double noise,
                                double jitter, double mean, const float* eps, int T, int Q, double tol,
                                const ciq_options* opt, float* out, ciq_info* info, ciq_stream_t stream) {
    if (n < 0 || n > CIQ_MAX_TRAIN || (n > 0 && (!Xtr || !y)) || !Xc || Nc < 1 || d < 1 || d > CIQ_MAX_DIM ||
        !lengthscales || !eps || !out || T < 1 || (kernel_type != CIQ_RBF && kernel_type != CIQ_MATERN52) ||
        !(outputscale > 0.0) || !std::isfinite(outputscale) || !(noise >= 0.0) || !std::isfinite(noise) ||
        !(jitter > 0.0) || !std::isfinite(jitter) || !std::isfinite(mean))
        return CIQ_ERR_ARG;
    for (int c = 0; c < d; ++c)
        if (!(lengthscales[c] > 0.0) || !std::isfinite(lengthscales[c])) return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    keep_pool_warm();
    const int64_t Npad = round_up(Nc, kRowPad);
    const int nn = (int)n;
    Arena ar;
    struct Buf {
        float *Xt, *Xc, *Xts, *Xcs, *Ct, *mu;
        double *ls, *M, *Kcx, *W, *a;
    };
    auto lay = [&](char* base) {
        ar = Arena{};
        ar.base = base;
        Buf b;
        b.Xt = ar.take<float>((size_t)std::max<int64_t>(n, 1) * d);
        b.Xc = ar.take<float>((size_t)Nc * d);
        b.Xts = ar.take<float>((size_t)std::max<int64_t>(n, 1) * d);
        b.Xcs = ar.take<float>((size_t)Nc * d);
        b.Ct = ar.take<float>((size_t)std::max(nn, 1) * Npad);
        b.mu = ar.take<float>((size_t)Npad);
        b.ls = ar.take<double>((size_t)d);
        b.M = ar.take<double>((size_t)std::max(nn, 1) * std::max(nn, 1));
        b.Kcx = ar.take<double>((size_t)std::max(nn, 1) * Npad);
        b.W = ar.take<double>((size_t)std::max(nn, 1) * std::max(nn, 1));
        b.a = ar.take<double>((size_t)std::max(nn, 1));
        return b;
    };
    lay(nullptr);
    const size_t need = ar.off + kAlign;
    char* base = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&base), need, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    const Buf b = lay(base);
    ciq_status rc = CIQ_OK;
    std::vector<double> M((size_t)nn * nn), lam(nn), U((size_t)nn * nn), W((size_t)nn * nn, 0.0), a(nn), yh(nn);
    int rk = 0;
    e = cudaMemcpyAsync(b.Xc, Xc, sizeof(float) * (size_t)Nc * d, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.ls, lengthscales, sizeof(double) * d, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_ard_scale(b.Xc, Nc, d, b.ls, b.Xcs, st);
    if (nn > 0) {
        if (e == cudaSuccess) e = cudaMemcpyAsync(b.Xt, Xtr, sizeof(float) * (size_t)n * d, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = launch_ard_scale(b.Xt, n, d, b.ls, b.Xts, st);
        // M = K_XX + sigma^2 I (FP64), to the host for its eigendecomposition.
        if (e == cudaSuccess)
            e = launch_kernel_block_f64(b.Xts, n, b.Xts, n, d, kernel_type, outputscale, noise, b.M, n, st);
        if (e == cudaSuccess) e = cudaMemcpyAsync(M.data(), b.M, sizeof(double) * M.size(), cudaMemcpyDeviceToHost, st);
        std::vector<float> yf(nn);
        if (e == cudaSuccess) e = cudaMemcpyAsync(yf.data(), y, sizeof(float) * nn, cudaMemcpyDefault, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        for (int i = 0; i < nn; ++i) yh[i] = (double)yf[i] - mean;
        if (e == cudaSuccess) {
            if (!symeig::eigh(nn, M.data(), lam.data(), U.data())) rc = CIQ_ERR_NAN;
        }
        if (e == cudaSuccess && rc == CIQ_OK) {
            // M = U diag(lambda) U^T; over the directions with lambda > 1e-13
            // max(lambda), W = U diag(lambda^{-1/2}) (n x rk) and C = K*X W, so
            // C C^T = K*X M^{-1} K_X*; a = W^T (y - m), so C a = K*X M^{-1} (y - m).
            const double lmax = lam[nn - 1];
            if (!(lmax > 0.0) || !std::isfinite(lmax)) rc = CIQ_ERR_NAN;
            for (int i = 0; rc == CIQ_OK && i < nn; ++i) {
                if (!(lam[i] > 1e-13 * lmax)) continue;
                const double f = 1.0 / std::sqrt(lam[i]);
                double sa = 0.0;
                for (int r = 0; r < nn; ++r) {
                    const double u = U[(size_t)r + (size_t)i * nn];
                    W[(size_t)r + (size_t)rk * nn] = u * f;
                    sa += u * yh[r];
                }
                a[rk] = sa * f;
                ++rk;
            }
        }
        if (e == cudaSuccess && rc == CIQ_OK && rk > 0) {
            e = cudaMemcpyAsync(b.W, W.data(), sizeof(double) * (size_t)nn * rk, cudaMemcpyHostToDevice, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(b.a, a.data(), sizeof(double) * rk, cudaMemcpyHostToDevice, st);
            // K*X in FP64 ([n][Npad], column m = training point m over the
            // candidates), then C^T = (K*X W)^T rounded once to FP32.
            if (e == cudaSuccess)
                e = launch_kernel_block_f64(b.Xcs, Nc, b.Xts, n, d, kernel_type, outputscale, 0.0, b.Kcx, Npad, st);
            if (e == cudaSuccess) e = launch_product_f64(b.Kcx, Npad, nn, b.W, rk, b.Ct, st);
            if (e == cudaSuccess) e = launch_posterior_mean(b.Ct, rk, Nc, Npad, b.a, mean, b.mu, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);       // the host vectors go out of scope
        }
    } else {
        if (e == cudaSuccess) e = launch_posterior_mean(b.Ct, 0, Nc, Npad, b.a, mean, b.mu, st);
    }
    if (e != cudaSuccess) rc = from_cuda(e);
    if (rc == CIQ_OK) {
        const ciq_kernel kc{kernel_type, 1.0, outputscale, jitter};       // candidates already divided by l_d
        const LrSpec lr{b.Ct, rk, b.mu};
        // With opt->precond_rank, a pivoted-Cholesky preconditioner of
        // COV* - jitter I (the device factors K** - C C^T).
        const int prk = opt ? opt->precond_rank : 0;
        const PcSpec pspec{nullptr, 0, prk};
        rc = solve<float>(b.Xcs, Nc, d, &kc, eps, T, Q, tol, opt, out, info, st, kOpSqrtIdentity, false, nullptr, 0,
                          nullptr, prk > 0 ? &pspec : nullptr, &lr);
    }
    cudaFreeAsync(base, st);
    cudaStreamSynchronize(st);
    if (rc != CIQ_OK && rc != CIQ_NOT_CONVERGED) cudaGetLastError();
    return rc;
}

size_t ciq_precond_workspace_bytes(int64_t N, int d, int T, int Q, int rank, const ciq_options* opt) {
    if (N < 1 || d < 1 || d > CIQ_MAX_DIM || T < 1 || Q < 1 || Q > CIQ_MAX_Q || rank < 1 || rank > kPcMaxRank ||
        rank > N)
        return 0;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    const bool prepass = !(o.quad_w && o.quad_t) && !(o.lmin > 0.0 && o.lmax > 0.0);
    const bool tc = o.precision != CIQ_PREC_FP32 && tc_supported(o.precision, d) && tc_padded_t(T) > 0;
    Plan<float> p = make_plan<float>(N, d, T, Q, o, prepass, tc, true);
    p.pc_rank = rank;
    p.nparts = p.nparts1 = (int)pc_row_tiles(p.Npad);
    p.layout(nullptr);
    return p.bytes;
}

size_t ciq_workspace_bytes(int64_t N, int d, int T, int Q, const ciq_options* opt) {
    if (N < 1 || d < 1 || d > CIQ_MAX_DIM || T < 1 || Q < 1 || Q > CIQ_MAX_Q) return 0;
    ciq_options o;
    ciq_default_options(&o);
    if (opt) o = *opt;
    const bool prepass = !(o.quad_w && o.quad_t) && !(o.lmin > 0.0 && o.lmax > 0.0);
    const bool tc = o.precision != CIQ_PREC_FP32 && tc_supported(o.precision, d) && tc_padded_t(T) > 0;
    Plan<float> p = make_plan<float>(N, d, T, Q, o, prepass, tc, true);
    return p.bytes;
}

ciq_status ciq_sqrt_batched(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                            ciq_info* infos, ciq_stream_t stream) {
    return solve_batched(probs, P, Q, tol, opt, infos, (cudaStream_t)stream, kOpSqrtIdentity);
}

ciq_status ciq_invsqrt_batched(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                               ciq_info* infos, ciq_stream_t stream) {
    return solve_batched(probs, P, Q, tol, opt, infos, (cudaStream_t)stream, kOpInvSqrt);
}

ciq_status ciq_sqrt_batched_learned(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                                    const float* theta, double margin, ciq_info* infos, int* fallback,
                                    ciq_stream_t stream) {
    return solve_batched_learned(probs, P, Q, tol, opt, theta, margin, infos, fallback, (cudaStream_t)stream,
                                 kOpSqrtIdentity);
}

ciq_status ciq_invsqrt_batched_learned(const ciq_problem* probs, int P, int Q, double tol, const ciq_options* opt,
                                       const float* theta, double margin, ciq_info* infos, int* fallback,
                                       ciq_stream_t stream) {
    return solve_batched_learned(probs, P, Q, tol, opt, theta, margin, infos, fallback, (cudaStream_t)stream,
                                 kOpInvSqrt);
}

// ------------------------------------------------------ learned predictor --
ciq_status ciq_mlp_features(const ciq_problem* probs, int P, float* F, ciq_stream_t stream) {
    if (!probs || P < 1 || P > CIQ_MAX_BATCH || !F || !device_accessible(F)) return CIQ_ERR_ARG;
    for (int p = 0; p < P; ++p)
        if (!probs[p].X || probs[p].N < 1 || probs[p].d < 1 || probs[p].d > CIQ_MAX_DIM ||
            !valid_kernel(&probs[p].kern) || !device_accessible(probs[p].X))
            return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    ciq_problem* pd = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&pd), sizeof(ciq_problem) * P, st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    e = cudaMemcpyAsync(pd, probs, sizeof(ciq_problem) * P, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_mlp_features(pd, P, F, st);
    cudaFreeAsync(pd, st);
    // The host array must stay readable until the copy is done.
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    return CIQ_OK;
}

ciq_status ciq_mlp_normaliser(const float* F, const float* Y, int n, float* theta, ciq_stream_t stream) {
    if (!F || !Y || !theta || n < 1 || !device_accessible(F) || !device_accessible(Y) || !device_accessible(theta))
        return CIQ_ERR_ARG;
    return from_cuda(launch_mlp_normaliser(F, Y, n, theta, (cudaStream_t)stream));
}

ciq_status ciq_mlp_init(float* theta, uint64_t seed, ciq_stream_t stream) {
    if (!theta || !device_accessible(theta)) return CIQ_ERR_ARG;
    return from_cuda(launch_mlp_init(theta, seed, (cudaStream_t)stream));
}

ciq_status ciq_mlp_loss_grad(const float* theta, const float* F, const float* Y, int n, double* loss, double* grad,
                             ciq_stream_t stream) {
    if (!theta || !F || !Y || !loss || !grad || n < 1 || !device_accessible(theta) || !device_accessible(F) ||
        !device_accessible(Y) || !device_accessible(grad))
        return CIQ_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    double* dl = nullptr;
    cudaError_t e = cudaMallocAsync(reinterpret_cast<void**>(&dl), sizeof(double), st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    e = launch_mlp_loss_grad(theta, F, Y, n, dl, grad, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(loss, dl, sizeof(double), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dl, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
    return CIQ_OK;
}

ciq_status ciq_mlp_train(float* theta, float* adam, const float* F, const float* Y, int n, int steps, int batch,
                         float lr, uint64_t seed, int first_step, float* losses, ciq_stream_t stream) {
    if (!theta || !adam || !F || !Y || n < 1 || steps < 0 || batch < 1 || batch > (1 << 20) || first_step < 1 ||
        !(lr > 0.f) || !device_accessible(theta) || !device_accessible(adam) || !device_accessible(F) ||
        !device_accessible(Y) || (losses && !device_accessible(losses)))
        return CIQ_ERR_ARG;
    if (steps == 0) return CIQ_OK;
    return from_cuda(launch_mlp_train(theta, adam, F, Y, n, steps, batch, lr, seed, first_step, losses,
                                      (cudaStream_t)stream));
}

ciq_status ciq_mlp_predict(const float* theta, const float* F, int n, float* out, int bf16, ciq_stream_t stream) {
    if (!theta || !F || !out || n < 1 || !device_accessible(theta) || !device_accessible(F) || !device_accessible(out))
        return CIQ_ERR_ARG;
    return from_cuda(launch_mlp_predict(theta, F, n, out, bf16 ? 1 : 0, (cudaStream_t)stream));
}

ciq_status ciq_invsqrt_vjp(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, const float* G,
                           int T, int Q, double tol, const ciq_options* opt, float* out, float* grad_B,
                           double* grad_theta, ciq_info* info, ciq_stream_t stream) {
    return solve_vjp(X, N, d, kern, B, G, T, Q, tol, opt, out, grad_B, grad_theta, info, (cudaStream_t)stream,
                     kOpInvSqrt);
}

ciq_status ciq_sqrt_vjp(const float* X, int64_t N, int d, const ciq_kernel* kern, const float* B, const float* G,
                        int T, int Q, double tol, const ciq_options* opt, float* out, float* grad_B,
                        double* grad_theta, ciq_info* info, ciq_stream_t stream) {
    return solve_vjp(X, N, d, kern, B, G, T, Q, tol, opt, out, grad_B, grad_theta, info, (cudaStream_t)stream,
                     kOpSqrtIdentity);
}

}  // extern "C"
