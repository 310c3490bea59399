// Bodies of the msMINRES recurrence and Lanczos pre-pass kernels (see
// krylov.cu), written against explicit block coordinates so that the
// single-problem kernels and the batched kernels (batched.cu) run the same code.
#pragma once

#include <math.h>

#include "krylov.cuh"
#include "spectral.cuh"

namespace ciq {
namespace {

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide FP64 sum (256 threads); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* red) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) red[warp] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < 8; ++w) r += red[w];
    return r;
}

template <typename R>
__device__ __forceinline__ R split_hi(double a) { return (R)a; }

template <typename R>
__device__ __forceinline__ void init_rhs_body(KrylovState<R> s, const R* B, int bx, int by) {
    __shared__ double red[8];
    const int k = bx, c = by;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
        const R v = i < s.N ? B[(int64_t)c * s.N + i] : (R)0;
        s.Bw[(int64_t)c * s.Npad + i] = v;
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) s.ynp[(int64_t)k * s.T + c] = acc;
}

template <typename R>
__device__ __forceinline__ void init_state_body(KrylovState<R> s, int bx, int by) {
    __shared__ double sh_inv;
    const int k = bx, c = by, tid = threadIdx.x;
    const int T = s.T, Q = s.Q;
    if (tid < 32) {
        double b2 = 0.0;
        for (int kk = tid; kk < s.nchunks; kk += 32) b2 += s.ynp[(int64_t)kk * T + c];
        b2 = warp_sum(b2);
        const double b1 = sqrt(b2);
        if (tid == 0) {
            sh_inv = b1 > 0.0 ? 1.0 / b1 : 0.0;
            if (k == 0) {
                s.beta1[c] = b1;
                s.beta[c] = 0.0;
                s.beta[T + c] = 0.0;
                s.status[c] = b1 > 0.0 ? kColRunning : kColExact;
                s.iters[c] = 0;
                s.brk[c] = 0;
            }
        }
        if (k == 0 && tid < Q) {
            for (int par = 0; par < 2; ++par) {
                double* g = s.giv + (((int64_t)par * Q + tid) * T + c) * 5;
                g[0] = 1.0; g[1] = 0.0; g[2] = 1.0; g[3] = 0.0; g[4] = b1;
            }
            s.phifinal[(int64_t)tid * T + c] = b1;
        }
    }
    __syncthreads();
    const R inv = (R)sh_inv;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    const int64_t col = (int64_t)c * s.Npad;
    for (int64_t i = i0 + tid; i < i1; i += 256) {
        s.QA[col + i] = s.Bw[col + i] * inv;
        s.QB[col + i] = (R)0;
        s.Y[col + i] = (R)0;
        s.Ylo[col + i] = (R)0;
    }
    for (int e = 0; s.D && e < 2 * Q; ++e) {
        R* d = s.D + ((int64_t)e * T + c) * s.Npad;
        for (int64_t i = i0 + tid; i < i1; i += 256) d[i] = (R)0;
    }
}

// BASIS: the stored-basis form (s.basis set).  Steps 1-3 are shared; the
// Givens factors of every shift are recorded instead of updating Q
// directions, and the vector work is q_{j+1} = (p - alpha q_j) / beta_{j+1}.
// The bodies take explicit block coordinates so that single solves and
// batched solves (batched.cu) run the same code.
template <typename R>
struct StepShared {
    double red[8][3];
    R co_delta[CIQ_MAX_Q], co_eps[CIQ_MAX_Q], co_invg[CIQ_MAX_Q], co_ct[CIQ_MAX_Q];
    R ahi, alo, invb;
    int skip;
};

// Steps 1-3 by one block of 256 threads for column c (k: the block's row
// chunk; chunk 0 writes the column's scalars).  Returns false when the
// column does no vector work this step.
template <typename R, bool BASIS>
__device__ __forceinline__ bool step_scalars(const KrylovState<R>& s, int j, int final_pass, int k, int c,
                                             StepShared<R>& sh) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int T = s.T, Q = s.Q;
    const int pin = j & 1, pout = (j + 1) & 1;
    const double* gin = s.giv + (int64_t)pin * Q * T * 5;
    double* gout = s.giv + (int64_t)pout * Q * T * 5;
    const double* w = s.nodes + kNodeW;
    const double* t = s.nodes + kNodeT;
    const double lmin = s.nodes[kNodeLmin];

    // 1. Decision for step j-1.
    if (warp == 0) {
        const int st = s.status[c];
        int code = kColRunning;
        if (st == kColRunning && j > 1) {
            if (s.brk[c]) {
                code = s.brk[c];
            } else if (s.tol > 0.0) {
                const double ph = lane < Q ? fabs(gin[((int64_t)lane * T + c) * 5 + 4]) : 0.0;
                if (s.stop_rule == CIQ_STOP_RESIDUAL) {
                    if (warp_max(ph) <= s.tol * s.beta1[c]) code = kColConverged;
                } else {
                    // Both square-root forms of the stored-basis rule weigh by w_q t_q.
                    const bool wt = BASIS ? s.op != kOpInvSqrt : s.op == kOpSqrtIdentity;
                    const double cq = lane < Q ? (wt ? w[lane] * t[lane] : w[lane]) : 0.0;
                    const double bound = warp_sum(lane < Q ? cq * ph / (t[lane] + lmin) : 0.0);
                    if constexpr (BASIS) {
                        // ||K^{1/2} b||^2 = b^T K b = ||b||^2 alpha_1; ||K^{-1/2} b||^2 >=
                        // ||b||^2 e_1^T T_{j-1}^{-1} e_1 (Gauss rule, from below).  With the
                        // (1 - 2 tol) factor the bound is also <= tol ||a_j|| at the stop.
                        // K (sum w_q x_q) is scaled by lambda_max, as in the oracle's reading.
                        const double* gs = s.gauss + ((int64_t)pin * T + c) * 4;
                        const double den2 = s.op == kOpInvSqrt ? gs[2] : gs[3];
                        const double den = (1.0 - 2.0 * s.tol) * s.beta1[c] * sqrt(fmax(den2, 0.0));
                        const double lm = s.nodes[kNodeLmax];
                        const double scale = s.op == kOpSqrtMvm && lm > 0.0 ? lm : 1.0;
                        if (bound * scale <= s.tol * den) code = kColConverged;
                    } else {
                        double yn = 0.0;
                        const double* yp = s.ynp + (int64_t)((j - 1) & 1) * s.nchunks * T;
                        for (int kk = lane; kk < s.nchunks; kk += 32) yn += yp[(int64_t)kk * T + c];
                        yn = warp_sum(yn);
                        if (bound <= s.tol * sqrt(yn)) code = kColConverged;
                    }
                }
            }
            if (final_pass && code == kColRunning) code = s.tol > 0.0 ? kColMaxIter : kColFixedIter;
        }
        const bool frozen = (st != kColRunning) || (code != kColRunning);
        if (lane == 0) sh.skip = frozen || final_pass;
        if (k == 0 && (frozen || final_pass)) {
            if (st == kColRunning) {
                if (lane < Q) s.phifinal[(int64_t)lane * T + c] = gin[((int64_t)lane * T + c) * 5 + 4];
                if (lane == 0) s.status[c] = code != kColRunning ? code : (s.tol > 0.0 ? kColMaxIter : kColFixedIter);
            }
            if (lane == 0 && !final_pass) {
                const int old = atomicAdd(&s.cnt[j], 1);
                if (old + 1 == T) atomicExch(s.all_done, 1);
            }
        }
    }
    __syncthreads();
    if (sh.skip) return false;

    // 2. alpha_j, beta_{j+1} from the MVM partial sums.  Every operand of
    // step 3 that does not depend on them is loaded first: the chain below is
    // FP64 (about 65 cycles per FMA, 430 per division, 670 per square root on
    // this part), and loads issued after its stores could not move above them.
    double c1 = 1.0, s1 = 0.0, c2 = 1.0, s2 = 0.0, ph = 0.0, tq = 0.0, cq = 0.0, beta_j = 0.0;
    double g_dp = 0.0, g_u2 = 0.0, g_S = 0.0, g_a1 = 0.0;
    if (warp == 0) {
        const int ql = lane < Q ? lane : 0;
        const double* g = gin + ((int64_t)ql * T + c) * 5;
        c1 = g[0]; s1 = g[1]; c2 = g[2]; s2 = g[3]; ph = g[4];
        tq = t[ql];
        cq = s.op == kOpSqrtIdentity ? w[ql] * tq : w[ql];
        beta_j = s.beta[pin * T + c];
        if constexpr (BASIS) {
            const double* gi = s.gauss + ((int64_t)pin * T + c) * 4;
            g_dp = gi[0]; g_u2 = gi[1]; g_S = gi[2]; g_a1 = gi[3];
        }
    }
    double qp = 0.0, pp = 0.0, qq = 0.0;
    for (int r = tid; r < s.nparts; r += 256) {
        const double* src = s.partials + ((int64_t)r * T + c) * 3;
        qp += src[0]; pp += src[1]; qq += src[2];
    }
    qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
    if (lane == 0) { sh.red[warp][0] = qp; sh.red[warp][1] = pp; sh.red[warp][2] = qq; }
    __syncthreads();
    if (warp == 0) {
        qp = lane < 8 ? sh.red[lane][0] : 0.0;
        pp = lane < 8 ? sh.red[lane][1] : 0.0;
        qq = lane < 8 ? sh.red[lane][2] : 0.0;
        qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
        const double alpha = qp;
        const double b2 = pp - 2.0 * alpha * qp + alpha * alpha * qq;
        const double beta_next = sqrt(fmax(b2, 0.0));
        const bool nan = !isfinite(alpha) || !isfinite(beta_next);
        const bool bd = nan || !(beta_next > s.breakdown_rtol * (fabs(alpha) + beta_j));
        const double bu = bd ? 0.0 : beta_next;
        const double inv_beta = bd ? 0.0 : 1.0 / beta_next;
        // 3. Givens QR update for every shift (one lane per shift; every lane
        // computes, lanes >= Q on shift 0's data and store nothing).
        const double abar = alpha + tq;
        const double eps = s2 * beta_j;
        const double dbar = c2 * beta_j;
        const double delta = c1 * dbar + s1 * abar;
        const double gbar = -s1 * dbar + c1 * abar;
        const double gamma = sqrt(gbar * gbar + bu * bu);
        const double ig = 1.0 / gamma;
        const double cj = gbar * ig, sj = bu * ig;
        const double tau = cj * ph;
        if (lane < Q) {
            sh.co_delta[lane] = (R)delta;
            sh.co_eps[lane] = (R)eps;
            sh.co_invg[lane] = (R)ig;
            sh.co_ct[lane] = (R)(cq * tau);
            if (k == 0) {
                double* go = gout + ((int64_t)lane * T + c) * 5;
                go[0] = cj; go[1] = sj; go[2] = c1; go[3] = s1; go[4] = -sj * ph;
                if constexpr (BASIS) {
                    // Column j of R_q (V_j = D_j R_q) and tau_j: x_q = V_J R_q^{-1} tau.
                    double* rc = s.rcoef + (((int64_t)(j - 1) * Q + lane) * T + c) * 4;
                    rc[0] = ig; rc[1] = delta; rc[2] = eps; rc[3] = tau;
                }
            }
        }
        if constexpr (BASIS) {
            // e_1^T T_j^{-1} e_1 by T_j = L D L^T: d_1 = alpha_1, d_k = alpha_k -
            // beta_k^2 / d_{k-1}, u_k^2 = u_{k-1}^2 beta_k^2 / d_{k-1}^2, sum u_k^2 / d_k.
            // A non-positive pivot (T_j not numerically SPD) ends the growth.
            double dk, u2, S, a1;
            if (j == 1) {
                dk = alpha; u2 = 1.0; S = 0.0; a1 = alpha;
            } else {
                S = g_S; a1 = g_a1;
                const double r = beta_j / g_dp;
                u2 = g_dp > 0.0 ? g_u2 * r * r : 0.0;
                dk = g_dp > 0.0 ? alpha - beta_j * r : -1.0;
            }
            if (dk > 0.0 && isfinite(dk) && isfinite(u2)) S += u2 / dk;
            else dk = -1.0;
            if (k == 0 && lane == 0) {
                double* go = s.gauss + ((int64_t)pout * T + c) * 4;
                go[0] = dk; go[1] = u2; go[2] = S; go[3] = a1;
            }
        }
        if (lane == 0) {
            const R ahi = (R)alpha;
            sh.ahi = ahi;
            sh.alo = (R)(alpha - (double)ahi);
            sh.invb = (R)inv_beta;
            sh.skip = nan;
            if (k == 0) {
                s.beta[pout * T + c] = bu;
                s.iters[c] = j;
                s.brk[c] = nan ? kColNaN : (bd ? kColExact : 0);
                if (s.tri && c == 0) {
                    s.tri[j - 1] = alpha;
                    s.tri[s.jmax + 1 + j] = bu;
                }
            }
        }
    }
    __syncthreads();
    if (sh.skip) return false;
    return true;
}

// Steps 4-5 for row chunk k of column c with the scalars of step_scalars.
template <typename R, bool BASIS>
__device__ __forceinline__ void step_vectors(const KrylovState<R>& s, int j, int k, int c, const StepShared<R>& sh) {
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    const int T = s.T, Q = s.Q;
    // 4. Vector updates for this chunk of rows.
    const R ahi = sh.ahi, alo = sh.alo, invb = sh.invb;
    const int64_t col = (int64_t)c * s.Npad;
    if constexpr (BASIS) {
        const int64_t vs = (int64_t)T * s.Npad;
        const R* qj = s.basis + (int64_t)j * vs + col;
        R* pn = s.basis + (int64_t)(j + 1) * vs + col;      // p in, q_{j+1} out
        const int64_t i0 = (int64_t)k * s.rows_per_chunk;
        const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
        if constexpr (sizeof(R) == 4) {
            const float4* q4 = reinterpret_cast<const float4*>(qj);
            float4* p4 = reinterpret_cast<float4*>(pn);
            // With a float-pair p its trailing part joins before the scaling.
            const float4* l4 = s.plo ? reinterpret_cast<const float4*>(s.plo + col) : nullptr;
            for (int64_t i4 = i0 / 4 + tid; i4 < i1 / 4; i4 += 256) {
                const float4 qv = q4[i4];
                const float4 pv = p4[i4];
                const float4 lv = l4 ? l4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
                const float qa[4] = {qv.x, qv.y, qv.z, qv.w}, pa[4] = {pv.x, pv.y, pv.z, pv.w};
                const float la[4] = {lv.x, lv.y, lv.z, lv.w};
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float t = fmaf(-(float)ahi, qa[e], pa[e]);
                    t = fmaf(-(float)alo, qa[e], t);
                    o[e] = (t + la[e]) * (float)invb;
                }
                p4[i4] = make_float4(o[0], o[1], o[2], o[3]);
            }
        } else {
            for (int64_t i = i0 + tid; i < i1; i += 256) {
                R t = fma(-ahi, qj[i], pn[i]);
                t = fma(-alo, qj[i], t);
                pn[i] = t * invb;
            }
        }
        return;
    }
    const R* q_j = ((j & 1) ? s.QA : s.QB) + col;
    R* pbuf = ((j & 1) ? s.QB : s.QA) + col;
    R* y = s.Y + col;
    R* ylo = s.Ylo + col;
    const R* b = s.Bw + col;
    const R sumw = (R)s.nodes[kNodeSumW];
    const int64_t dstride = (int64_t)T * s.Npad;
    R* d_prev = s.D + (int64_t)((j - 1) & 1) * Q * dstride + col;   // d_{j-1}
    R* d_old = s.D + (int64_t)(j & 1) * Q * dstride + col;          // d_{j-2}, overwritten by d_j
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    double ysq = 0.0;
    if constexpr (sizeof(R) == 4) {
        // FP32: four consecutive rows per thread with 16-byte loads and
        // stores (row chunks and the padded leading dimension are multiples
        // of 128, so a group of four never straddles either).
        constexpr int QB = 4;                  // shifts whose directions are loaded together
        const float4* q4 = reinterpret_cast<const float4*>(q_j);
        float4* p4 = reinterpret_cast<float4*>(pbuf);
        float4* y4 = reinterpret_cast<float4*>(y);
        float4* l4 = reinterpret_cast<float4*>(ylo);
        const float4* b4 = reinterpret_cast<const float4*>(b);
        // With a float-pair p its trailing part joins before the scaling.
        const float4* pl4 = s.plo ? reinterpret_cast<const float4*>(s.plo + col) : nullptr;
        const float4* dp4 = reinterpret_cast<const float4*>(d_prev);
        float4* do4 = reinterpret_cast<float4*>(d_old);
        const int64_t ds4 = dstride / 4;
        // ||a_j||^2 of this thread's rows in FP32 (a few dozen terms; the
        // stopping rule needs a few digits), converted to FP64 once: FP64
        // runs at a few operations per clock per SM on this part.
        float ysqf = 0.f;
        for (int64_t i4 = i0 / 4 + tid; i4 < i1 / 4; i4 += 256) {
            const float4 qv = q4[i4];
            const float4 pv = p4[i4];
            const float4 yv4 = y4[i4];
            const float4 lv4 = l4[i4];
            const float4 bv4 = s.op == kOpSqrtIdentity ? b4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 plv = pl4 ? pl4[i4] : make_float4(0.f, 0.f, 0.f, 0.f);
            float acc[4] = {0.f, 0.f, 0.f, 0.f};
            const float qa[4] = {qv.x, qv.y, qv.z, qv.w};
            for (int q0 = 0; q0 < Q; q0 += QB) {
                float4 dpv[QB], dqv[QB];
                const float4* pp = dp4 + (int64_t)q0 * ds4 + i4;
                const float4* po = do4 + (int64_t)q0 * ds4 + i4;
#pragma unroll
                for (int u = 0; u < QB; ++u) {
                    dpv[u] = q0 + u < Q ? pp[u * ds4] : make_float4(0.f, 0.f, 0.f, 0.f);
                    dqv[u] = q0 + u < Q ? po[u * ds4] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < QB; ++u) {
                    if (q0 + u >= Q) break;
                    const int qq2 = q0 + u;
                    const float de = sh.co_delta[qq2], ep = sh.co_eps[qq2], ig = sh.co_invg[qq2], ct = sh.co_ct[qq2];
                    const float pa[4] = {dpv[u].x, dpv[u].y, dpv[u].z, dpv[u].w};
                    const float oa[4] = {dqv[u].x, dqv[u].y, dqv[u].z, dqv[u].w};
                    float dn[4];
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        dn[e] = (qa[e] - de * pa[e] - ep * oa[e]) * ig;
                        acc[e] = fmaf(ct, dn[e], acc[e]);
                    }
                    do4[(int64_t)qq2 * ds4 + i4] = make_float4(dn[0], dn[1], dn[2], dn[3]);
                }
            }
            const float pa[4] = {pv.x, pv.y, pv.z, pv.w};
            const float ya[4] = {yv4.x, yv4.y, yv4.z, yv4.w};
            const float la[4] = {lv4.x, lv4.y, lv4.z, lv4.w};
            const float ba[4] = {bv4.x, bv4.y, bv4.z, bv4.w};
            const float pla[4] = {plv.x, plv.y, plv.z, plv.w};
            float pn[4], ys[4], yl[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float t = fmaf(-(float)ahi, qa[e], pa[e]);
                t = fmaf(-(float)alo, qa[e], t);
                pn[e] = (t + pla[e]) * (float)invb;
                // y += acc as a (leading, trailing) pair (Knuth's 2Sum).
                const float sum = ya[e] + acc[e];
                const float bp = sum - ya[e];
                const float err = (ya[e] - (sum - bp)) + (acc[e] - bp);
                ys[e] = sum;
                yl[e] = la[e] + err;
                const float yv = sum + yl[e];
                const float est = s.op == kOpSqrtIdentity ? (float)sumw * ba[e] - yv : yv;
                ysqf = fmaf(est, est, ysqf);
            }
            p4[i4] = make_float4(pn[0], pn[1], pn[2], pn[3]);
            y4[i4] = make_float4(ys[0], ys[1], ys[2], ys[3]);
            l4[i4] = make_float4(yl[0], yl[1], yl[2], yl[3]);
        }
        ysq = (double)ysqf;
    } else {
        constexpr int QB = 8;                  // shifts whose directions are loaded together
        for (int64_t i = i0 + tid; i < i1; i += 256) {
            // Every load of the row is issued before any store (the compiler
            // cannot move a load above a store that may alias it), so the HBM
            // latency is paid once per block of QB shifts rather than per shift.
            const R q = q_j[i];
            R pn = pbuf[i];
            const R yh = y[i];
            const R ylo_i = ylo[i];
            const R b_i = s.op == kOpSqrtIdentity ? b[i] : (R)0;
            R acc = (R)0;
            for (int q0 = 0; q0 < Q; q0 += QB) {
                R dp[QB], dq[QB];
                const R* pp = d_prev + (int64_t)q0 * dstride + i;
                const R* po = d_old + (int64_t)q0 * dstride + i;
    #pragma unroll
                for (int u = 0; u < QB; ++u) {
                    dp[u] = q0 + u < Q ? pp[u * dstride] : (R)0;
                    dq[u] = q0 + u < Q ? po[u * dstride] : (R)0;
                }
    #pragma unroll
                for (int u = 0; u < QB; ++u) {
                    if (q0 + u >= Q) break;
                    const int qq2 = q0 + u;
                    const R dn = (q - sh.co_delta[qq2] * dp[u] - sh.co_eps[qq2] * dq[u]) * sh.co_invg[qq2];
                    d_old[(int64_t)qq2 * dstride + i] = dn;
                    acc = fma(sh.co_ct[qq2], dn, acc);
                }
            }
            pn = fma(-ahi, q, pn);
            pn = fma(-alo, q, pn);
            pbuf[i] = pn * invb;
            // y += acc as a (leading, trailing) pair: Knuth's 2Sum error term goes
            // to the trailing part, so the sum keeps ~2x R's precision.  The K^{1/2}
            // identity form later subtracts y from (sum w) b, which cancels.
            const R sum = yh + acc;
            const R bp = sum - yh;
            const R err = (yh - (sum - bp)) + (acc - bp);
            const R yl = ylo_i + err;
            y[i] = sum;
            ylo[i] = yl;
            const R yv = sum + yl;
            const R est = s.op == kOpSqrtIdentity ? sumw * b_i - yv : yv;
            ysq += (double)est * (double)est;
        }
    }
    // 5. Partial ||a_j||^2 for the next decision.
    ysq = warp_sum(ysq);
    __shared__ double red2[8];
    if (lane == 0) red2[warp] = ysq;
    __syncthreads();
    if (tid == 0) {
        double r = 0.0;
        for (int ww = 0; ww < 8; ++ww) r += red2[ww];
        s.ynp[((int64_t)(j & 1) * s.nchunks + k) * T + c] = r;
    }
}

// The step in two launches: one block per column computes the scalars once
// and publishes them (sco); the row-chunk blocks only read them.  The FP64
// work is then done once per column instead of once per row chunk, where
// the chunks of one SM would queue on its FP64 pipe.
template <typename R, bool BASIS>
__device__ __forceinline__ void step_scalar_body(KrylovState<R> s, int j, int final_pass, int c) {
    if (!final_pass && *s.all_done) return;
    __shared__ StepShared<R> sh;
    const bool go = step_scalars<R, BASIS>(s, j, final_pass, 0, c, sh);
    if (final_pass) return;
    R* dst = s.sco + (int64_t)c * kScoStride;
    const int tid = threadIdx.x;
    if (tid == 0) {
        dst[0] = go ? (R)0 : (R)1;
        dst[1] = sh.ahi; dst[2] = sh.alo; dst[3] = sh.invb;
    }
    if (go && !BASIS && tid < s.Q) {
        dst[4 + tid] = sh.co_delta[tid];
        dst[4 + CIQ_MAX_Q + tid] = sh.co_eps[tid];
        dst[4 + 2 * CIQ_MAX_Q + tid] = sh.co_invg[tid];
        dst[4 + 3 * CIQ_MAX_Q + tid] = sh.co_ct[tid];
    }
}

template <typename R, bool BASIS>
__device__ __forceinline__ void step_vector_body(KrylovState<R> s, int j, int k, int c) {
    if (*s.all_done) return;
    const R* src = s.sco + (int64_t)c * kScoStride;
    if (src[0] != (R)0) return;
    __shared__ StepShared<R> sh;
    const int tid = threadIdx.x;
    if (tid == 0) { sh.ahi = src[1]; sh.alo = src[2]; sh.invb = src[3]; }
    if (!BASIS && tid < s.Q) {
        sh.co_delta[tid] = src[4 + tid];
        sh.co_eps[tid] = src[4 + CIQ_MAX_Q + tid];
        sh.co_invg[tid] = src[4 + 2 * CIQ_MAX_Q + tid];
        sh.co_ct[tid] = src[4 + 3 * CIQ_MAX_Q + tid];
    }
    __syncthreads();
    step_vectors<R, BASIS>(s, j, k, c, sh);
}

template <typename R>
__device__ __forceinline__ void combine_body(KrylovState<R> s, R* out, int bx, int by) {
    const int64_t i = (int64_t)bx * blockDim.x + threadIdx.x;
    const int c = by;
    if (i >= s.N) return;
    const int64_t src = (int64_t)c * s.Npad + i;
    const double yv = (double)s.Y[src] + (double)s.Ylo[src];
    double v = yv;
    if (s.op == kOpSqrtIdentity) v = s.nodes[kNodeSumW] * (double)s.Bw[src] - yv;
    if (s.op == kOpSqrtMvm) s.Y[src] = (R)yv;      // folded into one vector for the final MVM
    out[(int64_t)c * s.N + i] = (R)v;
}

// Stored-basis form, part 1: one warp per column, one lane per shift.  Back
// substitution R_q y_q = tau_q (R_q upper triangular with gamma_j, delta_{j+1},
// eps_{j+2} on its three diagonals) from the last step down, in FP64, and the
// CIQ combination sum_q c_q y_q(j) of every basis vector's coefficient.  The
// factors come through shared memory 32 steps at a time and the sums over
// shifts are taken after each group, so the FP64 chain carries only
// y_j = ((tau_j - eps_{j+2} y_{j+2}) - delta_{j+1} y_{j+1}) / gamma_j.
template <typename R>
__device__ __forceinline__ void basis_backsub_body(KrylovState<R> s, int c) {
    constexpr int CH = 32;
    __shared__ double co[CH][CIQ_MAX_Q][4];
    __shared__ double cy[CH][CIQ_MAX_Q + 1];
    const int lane = threadIdx.x & 31, T = s.T, Q = s.Q;
    const int J = s.iters[c];
    const double* w = s.nodes + kNodeW;
    const double* t = s.nodes + kNodeT;
    const bool on = lane < Q;
    const double cq = on ? (s.op == kOpSqrtIdentity ? w[lane] * t[lane] : w[lane]) : 0.0;
    double y1 = 0.0, y2 = 0.0, dl1 = 0.0, ep1 = 0.0, ep2 = 0.0;   // y_{j+1}, y_{j+2}, delta_{j+1}, eps_{j+1}, eps_{j+2}
    for (int jt = J; jt >= 1; jt -= CH) {                // steps jt, jt - 1, ..., jt - n + 1
        const int n = min(CH, jt);
        __syncwarp();
        if (on) {
            // Lane q copies its own factors; unrolled so that eight steps' loads
            // are in flight at once (the shared stores cannot alias them).
#pragma unroll 8
            for (int u = 0; u < n; ++u) {
                const double2* src =
                    reinterpret_cast<const double2*>(s.rcoef + (((int64_t)(jt - u - 1) * Q + lane) * T + c) * 4);
                const double2 a = src[0], b = src[1];
                co[u][lane][0] = a.x; co[u][lane][1] = a.y; co[u][lane][2] = b.x; co[u][lane][3] = b.y;
            }
        }
        __syncwarp();
        if (on) {
            for (int u = 0; u < n; ++u) {
                const double invg = co[u][lane][0], de = co[u][lane][1], ep = co[u][lane][2], tau = co[u][lane][3];
                const double y = fma(-dl1, y1, fma(-ep2, y2, tau)) * invg;
                ep2 = ep1; ep1 = ep; dl1 = de; y2 = y1; y1 = y;
                cy[u][lane] = cq * y;
                if (s.ycoef) s.ycoef[((int64_t)(jt - u) * Q + lane) * T + c] = y;
            }
        }
        __syncwarp();
        if (lane < n) {
            double tot = 0.0;
            for (int q = 0; q < Q; ++q) tot += cy[lane][q];
            s.bco[(int64_t)(jt - lane) * T + c] = tot;
        }
    }
}

// Stored-basis form, part 2: one block per (row chunk, column).  The sum
// sum_j coef_j q_j runs over the basis once, in FP32 with the coefficient split
// in two floats, the exact product error (FMA) and Knuth's 2Sum, so that the
// K^{1/2} identity form's cancellation against (sum w) b keeps FP32 accuracy.
template <typename R>
__device__ __forceinline__ void basis_combine_body(KrylovState<R> s, R* out, int final_j, int k, int c) {
    __shared__ float2 cof[256];
    __shared__ double cod[256];
    __shared__ double red[8];
    const int tid = threadIdx.x, T = s.T;
    const int J = s.iters[c];
    const int64_t vs = (int64_t)T * s.Npad;
    const int64_t col = (int64_t)c * s.Npad;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    const double sumw = s.nodes[kNodeSumW];
    constexpr int RPT = sizeof(R) == 4 ? 4 : 1;           // rows per thread
    double ysq = 0.0;
    for (int64_t base = i0; base < i1; base += 256 * RPT) {
        const int64_t i = base + (int64_t)RPT * tid;
        const bool act = i < i1;
        float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
        double acc = 0.0;
        for (int jb = 1; jb <= J; jb += 256) {
            const int nj = min(256, J - jb + 1);
            __syncthreads();
            if (tid < nj) {
                const double cf = s.bco[(int64_t)(jb + tid) * T + c];
                const float h = (float)cf;
                cof[tid] = make_float2(h, (float)(cf - (double)h));
                cod[tid] = cf;
            }
            __syncthreads();
            if (!act) continue;
            const R* vp = s.basis + (int64_t)jb * vs + col + i;
            if constexpr (sizeof(R) == 4) {
#pragma unroll 4
                for (int u = 0; u < nj; ++u) {
                    const float2 cf = cof[u];
                    const float4 v4 = *reinterpret_cast<const float4*>(vp + (int64_t)u * vs);
                    const float va[4] = {v4.x, v4.y, v4.z, v4.w};
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const float pr = cf.x * va[e];
                        const float pe = fmaf(cf.x, va[e], -pr) + cf.y * va[e];
                        const float sm = hi[e] + pr;
                        const float bp = sm - hi[e];
                        lo[e] += ((hi[e] - (sm - bp)) + (pr - bp)) + pe;
                        hi[e] = sm;
                    }
                }
            } else {
                for (int u = 0; u < nj; ++u) acc = fma(cod[u], (double)vp[(int64_t)u * vs], acc);
            }
        }
        if (!act) continue;
#pragma unroll
        for (int e = 0; e < RPT; ++e) {
            const int64_t r = i + e;
            const double sv = sizeof(R) == 4 ? (double)hi[e] + (double)lo[e] : acc;
            double v = sv;
            if (s.op == kOpSqrtIdentity) v = sumw * (double)s.Bw[col + r] - sv;
            if (s.op == kOpSqrtMvm) s.Y[col + r] = (R)sv;
            else if (r < s.N) out[(int64_t)c * s.N + r] = (R)v;
            ysq += v * v;
        }
    }
    ysq = warp_sum(ysq);
    if ((tid & 31) == 0) red[tid >> 5] = ysq;
    __syncthreads();
    if (tid == 0) {
        double r = 0.0;
        for (int ww = 0; ww < 8; ++ww) r += red[ww];
        s.ynp[((int64_t)(final_j & 1) * s.nchunks + k) * T + c] = r;
    }
}

// summary[0] max iters, [1] min iters, [2] converged columns, [3] max |phibar|/||b||,
// [4] max errbound/||a||, [5] worst status, [6] NaN columns.
template <typename R>
__device__ __forceinline__ void summary_body(KrylovState<R> s, int final_j, int bx, int by) {
    if (threadIdx.x != 0) return;
    const int T = s.T, Q = s.Q;
    const double* w = s.nodes + kNodeW;
    const double* t = s.nodes + kNodeT;
    const double lmin = s.nodes[kNodeLmin];
    int itmax = 0, itmin = 1 << 30, conv = 0, nans = 0, worst = 0;
    double rmax = 0.0, emax = 0.0;
    const double* yp = s.ynp + (int64_t)(final_j & 1) * s.nchunks * T;
    for (int c = 0; c < T; ++c) {
        const int it = s.iters[c];
        itmax = max(itmax, it);
        itmin = min(itmin, it);
        const int st = s.status[c];
        if (st == kColConverged || st == kColExact) ++conv;
        if (st == kColNaN) ++nans;
        worst = max(worst, st);
        const double b1 = s.beta1[c];
        double bound = 0.0, rm = 0.0;
        for (int q = 0; q < Q; ++q) {
            const double ph = fabs(s.phifinal[(int64_t)q * T + c]);
            rm = fmax(rm, ph);
            const double cq = s.op == kOpSqrtIdentity ? w[q] * t[q] : w[q];
            bound += cq * ph / (t[q] + lmin);
        }
        if (b1 > 0.0) rmax = fmax(rmax, rm / b1);
        double yn = 0.0;
        for (int kk = 0; kk < s.nchunks; ++kk) yn += yp[(int64_t)kk * T + c];
        if (yn > 0.0) emax = fmax(emax, bound / sqrt(yn));
    }
    s.summary[0] = itmax;
    s.summary[1] = T > 0 ? itmin : 0;
    s.summary[2] = conv;
    s.summary[3] = rmax;
    s.summary[4] = emax;
    s.summary[5] = worst;
    s.summary[6] = nans;
}

// ---------------------------------------------------------------- pre-pass --
__device__ __forceinline__ double splitmix_uniform(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z = z ^ (z >> 31);
    return (double)(z >> 11) * 0x1.0p-53;
}

template <typename R>
__device__ __forceinline__ void lanczos_init_a_body(LanczosState<R> s, const R* start, uint64_t seed, int bx, int by) {
    __shared__ double red[8];
    const int k = bx;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    double acc = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) {
        R v = (R)0;
        if (i < s.N) v = start ? start[i] : (R)(2.0 * splitmix_uniform(seed, (uint64_t)i) - 1.0);
        s.LA[i] = v;
        s.LB[i] = (R)0;
        acc += (double)v * (double)v;
    }
    acc = block_sum(acc, red);
    if (threadIdx.x == 0) s.ynp[k] = acc;
}

template <typename R>
__device__ __forceinline__ void lanczos_init_b_body(LanczosState<R> s, int bx, int by) {
    __shared__ double sh_inv;
    const int k = bx;
    if (threadIdx.x < 32) {
        double b2 = 0.0;
        for (int kk = threadIdx.x; kk < s.nchunks; kk += 32) b2 += s.ynp[kk];
        b2 = warp_sum(b2);
        if (threadIdx.x == 0) {
            const double b1 = sqrt(b2);
            sh_inv = b1 > 0.0 ? 1.0 / b1 : 0.0;
            if (k == 0) {
                s.beta[0] = b1;
                s.bpar[0] = 0.0;
                s.bpar[1] = 0.0;
                *s.jeff = 0;
                *s.done = b1 > 0.0 ? 0 : 1;
            }
        }
    }
    __syncthreads();
    const R inv = (R)sh_inv;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    for (int64_t i = i0 + threadIdx.x; i < i1; i += 256) s.LA[i] *= inv;
}

template <typename R>
__device__ __forceinline__ void lanczos_step_body(LanczosState<R> s, int j, int bx, int by) {
    if (*s.done) return;
    __shared__ double red[8][3];
    __shared__ R sh_ahi, sh_alo, sh_invb;
    const int k = bx, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double qp = 0.0, pp = 0.0, qq = 0.0;
    for (int r = tid; r < s.nparts; r += 256) {
        qp += s.partials[r * 3 + 0]; pp += s.partials[r * 3 + 1]; qq += s.partials[r * 3 + 2];
    }
    qp = warp_sum(qp); pp = warp_sum(pp); qq = warp_sum(qq);
    if (lane == 0) { red[warp][0] = qp; red[warp][1] = pp; red[warp][2] = qq; }
    __syncthreads();
    if (tid == 0) {
        qp = pp = qq = 0.0;
        for (int w = 0; w < 8; ++w) { qp += red[w][0]; pp += red[w][1]; qq += red[w][2]; }
        const double alpha = qp;
        const double beta_next = sqrt(fmax(pp - 2.0 * alpha * qp + alpha * alpha * qq, 0.0));
        const double beta_j = s.bpar[j & 1];
        const bool bd = !isfinite(alpha) || !(beta_next > 1e-12 * (fabs(alpha) + beta_j));
        const R ahi = (R)alpha;
        sh_ahi = ahi;
        sh_alo = (R)(alpha - (double)ahi);
        sh_invb = bd ? (R)0 : (R)(1.0 / beta_next);
        if (k == 0) {
            s.alpha[j - 1] = alpha;
            s.beta[j] = bd ? 0.0 : beta_next;
            s.bpar[(j + 1) & 1] = bd ? 0.0 : beta_next;
            *s.jeff = j;
            if (bd) *s.done = 1;
        }
    }
    __syncthreads();
    const R ahi = sh_ahi, alo = sh_alo, invb = sh_invb;
    const R* q_j = (j & 1) ? s.LA : s.LB;
    R* pbuf = (j & 1) ? s.LB : s.LA;
    const int64_t i0 = (int64_t)k * s.rows_per_chunk;
    const int64_t i1 = min(i0 + s.rows_per_chunk, s.Npad);
    for (int64_t i = i0 + tid; i < i1; i += 256) {
        R pn = pbuf[i];
        const R q = q_j[i];
        pn = fma(-ahi, q, pn);
        pn = fma(-alo, q, pn);
        pbuf[i] = pn * invb;
    }
}

template <typename R>
__device__ __forceinline__ void bounds_nodes_body(LanczosState<R> s, double* nodes, int Q, double noise,
                                    double lmax_margin, double lmin_div, int bx, int by) {
    if (threadIdx.x != 0 || bx != 0) return;
    const int J = *s.jeff;
    double th_min = 0.0, th_max = 0.0;
    if (J >= 1) {
        th_min = tridiag_extreme(s.alpha, s.beta, J, false);
        th_max = tridiag_extreme(s.alpha, s.beta, J, true);
    }
    const double lmax = lmax_margin * th_max;
    double lmin = noise > 0.0 ? noise : th_min / lmin_div;
    if (!(lmin > 0.0)) lmin = 1e-300;
    double w[CIQ_MAX_Q], t[CIQ_MAX_Q];
    const double lmax_u = fmax(lmax, lmin);
    quad_nodes(lmin, lmax_u, Q, w, t);
    double sw = 0.0;
    for (int q = 0; q < CIQ_MAX_Q; ++q) {
        nodes[kNodeW + q] = q < Q ? w[q] : 0.0;
        nodes[kNodeT + q] = q < Q ? t[q] : 0.0;
        if (q < Q) sw += w[q];
    }
    nodes[kNodeLmin] = lmin;
    nodes[kNodeLmax] = lmax_u;
    nodes[kNodeRitzMin] = th_min;
    nodes[kNodeRitzMax] = th_max;
    nodes[kNodeSumW] = sw;
    nodes[kNodeLanczosSteps] = J;
}

// Nodes for given bounds (one thread).
__device__ __forceinline__ void nodes_from_bounds_body(double* nodes, int Q, double lmin, double lmax) {
    double w[CIQ_MAX_Q], t[CIQ_MAX_Q];
    quad_nodes(lmin, lmax, Q, w, t);
    double sw = 0.0;
    for (int q = 0; q < CIQ_MAX_Q; ++q) {
        nodes[kNodeW + q] = q < Q ? w[q] : 0.0;
        nodes[kNodeT + q] = q < Q ? t[q] : 0.0;
        if (q < Q) sw += w[q];
    }
    nodes[kNodeLmin] = lmin;
    nodes[kNodeLmax] = lmax;
    nodes[kNodeRitzMin] = 0.0;
    nodes[kNodeRitzMax] = 0.0;
    nodes[kNodeSumW] = sw;
    nodes[kNodeLanczosSteps] = 0.0;
}

}  // namespace
}  // namespace ciq
