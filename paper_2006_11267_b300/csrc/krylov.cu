// msMINRES recurrence and Lanczos bound pre-pass (App. B.2, App. C).
//
// One msMINRES iteration is the kernel MVM with its Lanczos epilogue
// (p = K q_j - beta_j q_{j-1} and FP64 partial sums of q.p, p.p, q.q) and
// the recurrence step, split in two launches: step_scalar (one block per
// column: steps 1-3) and step_vector (one block per row chunk and column:
// steps 4-5).  Batched solves launch the same two bodies over their work
// lists, so their results equal single solves bit for bit.
//
//  1. decide whether the column stopped after step j-1 (stop rule, breakdown);
//  2. alpha_j = q.p and beta_{j+1}^2 = p.p - 2 alpha q.p + alpha^2 q.q in FP64
//     from the MVM partial sums (reduced in one fixed order);
//  3. per shift t_q, one lane each: the Givens update of T_j + t_q I
//     (Eq. minres_qr_shifted, standard Paige-Saunders form) in FP64;
//  4. per row: q_{j+1} = (p - alpha q_j) / beta_{j+1} (alpha split in two
//     floats so the cancellation keeps FP32 accuracy), d_j^{(q)} =
//     (q_j - delta d_{j-1} - eps d_{j-2}) / gamma for every shift, and the
//     CIQ sum y += sum_q c_q tau_q d_j^{(q)} (Eq. contour_integral_quad),
//     which never stores the Q solutions themselves;
//  5. partial ||a_j||^2 of the current estimate for the error-bound rule.
//
// Scalars that one launch reads and the next writes are double-buffered by
// the parity of j, so blocks of one launch never race.
//
// Stored-basis form: step 4 shrinks to q_{j+1} = (p - alpha q_j) / beta_{j+1}
// in the basis slot j + 1 (read 2, write 1 vector instead of 3Q + 4), and
// step 3 records gamma, delta, eps, tau of every shift.  After the last step,
// basis_backsub solves R_q y_q = tau_q in FP64 and basis_combine forms
// sum_j (sum_q c_q y_q(j)) q_j in one pass over the basis: the iterates of
// Eq. minres_qr_shifted without the per-step direction traffic.
#include <math.h>

#include "krylov.cuh"
#include "krylov_body.cuh"
#include "spectral.cuh"

namespace ciq {

namespace {

template <typename R>
__global__ void __launch_bounds__(256) init_rhs_kernel(KrylovState<R> s, const R* B) {
    init_rhs_body<R>(s, B, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(256) init_state_kernel(KrylovState<R> s) {
    init_state_body<R>(s, blockIdx.x, blockIdx.y);
}


template <typename R, bool BASIS>
__global__ void __launch_bounds__(256) step_scalar_kernel(KrylovState<R> s, int j, int final_pass) {
    step_scalar_body<R, BASIS>(s, j, final_pass, blockIdx.x);
}

// Three blocks per SM (at most 85 registers): the vector update is HBM-bound
// and needs the resident threads more than registers.
template <typename R, bool BASIS>
__global__ void __launch_bounds__(256, 3) step_vector_kernel(KrylovState<R> s, int j) {
    step_vector_body<R, BASIS>(s, j, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(32) basis_backsub_kernel(KrylovState<R> s) {
    basis_backsub_body<R>(s, blockIdx.x);
}

template <typename R>
__global__ void __launch_bounds__(256) basis_combine_kernel(KrylovState<R> s, R* out, int final_j) {
    basis_combine_body<R>(s, out, final_j, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void combine_kernel(KrylovState<R> s, R* out) {
    combine_body<R>(s, out, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void summary_kernel(KrylovState<R> s, int final_j) {
    summary_body<R>(s, final_j, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(256) lanczos_init_a(LanczosState<R> s, const R* start, uint64_t seed) {
    lanczos_init_a_body<R>(s, start, seed, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(256) lanczos_init_b(LanczosState<R> s) {
    lanczos_init_b_body<R>(s, blockIdx.x, blockIdx.y);
}

template <typename R>
__global__ void __launch_bounds__(256) lanczos_step_kernel(LanczosState<R> s, int j) {
    lanczos_step_body<R>(s, j, blockIdx.x, blockIdx.y);
}

__global__ void nodes_from_bounds_kernel(double* nodes, int Q, double lmin, double lmax) {
    if (threadIdx.x == 0 && blockIdx.x == 0) nodes_from_bounds_body(nodes, Q, lmin, lmax);
}

template <typename R>
__global__ void bounds_nodes_kernel(LanczosState<R> s, double* nodes, int Q, double noise,
                                    double lmax_margin, double lmin_div) {
    bounds_nodes_body<R>(s, nodes, Q, noise, lmax_margin, lmin_div, blockIdx.x, blockIdx.y);
}

}  // namespace

template <typename R>
cudaError_t launch_init_rhs(const KrylovState<R>& s, const R* B, cudaStream_t st) {
    init_rhs_kernel<R><<<dim3(s.nchunks, s.T), 256, 0, st>>>(s, B);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_init_state(const KrylovState<R>& s, cudaStream_t st) {
    init_state_kernel<R><<<dim3(s.nchunks, s.T), 256, 0, st>>>(s);
    return cudaGetLastError();
}
// Resident recurrence blocks on the whole GPU (row chunks are sized to it).
int step_blocks_per_wave() {
    static int w = 0;
    if (w == 0) {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, step_vector_kernel<float, false>, 256, 0) != cudaSuccess ||
            sms <= 0 || per_sm <= 0) {
            cudaGetLastError();
            return 148 * 3;
        }
        w = sms * per_sm;
    }
    return w;
}

template <typename R>
cudaError_t launch_msminres_step(const KrylovState<R>& s, int j, bool final_pass, cudaStream_t st, bool vector_part) {
    // One block per column for the scalars, then the row chunks (none after
    // the final decision pass).
    const int fp = final_pass ? 1 : 0;
    if (s.basis) step_scalar_kernel<R, true><<<s.T, 256, 0, st>>>(s, j, fp);
    else step_scalar_kernel<R, false><<<s.T, 256, 0, st>>>(s, j, fp);
    if (!final_pass && vector_part) {
        const dim3 grid(s.nchunks, s.T);
        if (s.basis) step_vector_kernel<R, true><<<grid, 256, 0, st>>>(s, j);
        else step_vector_kernel<R, false><<<grid, 256, 0, st>>>(s, j);
    }
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_basis_combine(const KrylovState<R>& s, R* out, int final_j, cudaStream_t st) {
    basis_backsub_kernel<R><<<s.T, 32, 0, st>>>(s);
    basis_combine_kernel<R><<<dim3(s.nchunks, s.T), 256, 0, st>>>(s, out, final_j);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_combine(const KrylovState<R>& s, R* out, cudaStream_t st) {
    combine_kernel<R><<<dim3((unsigned)((s.N + 255) / 256), s.T), 256, 0, st>>>(s, out);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_summary(const KrylovState<R>& s, int final_j, cudaStream_t st) {
    summary_kernel<R><<<1, 32, 0, st>>>(s, final_j);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_lanczos_init(const LanczosState<R>& s, const R* start, uint64_t seed, cudaStream_t st) {
    lanczos_init_a<R><<<s.nchunks, 256, 0, st>>>(s, start, seed);
    lanczos_init_b<R><<<s.nchunks, 256, 0, st>>>(s);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_lanczos_step(const LanczosState<R>& s, int j, cudaStream_t st) {
    lanczos_step_kernel<R><<<s.nchunks, 256, 0, st>>>(s, j);
    return cudaGetLastError();
}
template <typename R>
cudaError_t launch_bounds_nodes(const LanczosState<R>& s, double* nodes, int Q, double noise,
                                double lmax_margin, double lmin_div, cudaStream_t st) {
    bounds_nodes_kernel<R><<<1, 32, 0, st>>>(s, nodes, Q, noise, lmax_margin, lmin_div);
    return cudaGetLastError();
}
cudaError_t launch_nodes_from_bounds(double* nodes, int Q, double lmin, double lmax, cudaStream_t st) {
    nodes_from_bounds_kernel<<<1, 32, 0, st>>>(nodes, Q, lmin, lmax);
    return cudaGetLastError();
}

#define CIQ_INSTANTIATE(R)                                                                          \
    template cudaError_t launch_init_rhs<R>(const KrylovState<R>&, const R*, cudaStream_t);           \
    template cudaError_t launch_init_state<R>(const KrylovState<R>&, cudaStream_t);                   \
    template cudaError_t launch_msminres_step<R>(const KrylovState<R>&, int, bool, cudaStream_t, bool); \
    template cudaError_t launch_combine<R>(const KrylovState<R>&, R*, cudaStream_t);                  \
    template cudaError_t launch_basis_combine<R>(const KrylovState<R>&, R*, int, cudaStream_t);       \
    template cudaError_t launch_summary<R>(const KrylovState<R>&, int, cudaStream_t);                 \
    template cudaError_t launch_lanczos_init<R>(const LanczosState<R>&, const R*, uint64_t, cudaStream_t); \
    template cudaError_t launch_lanczos_step<R>(const LanczosState<R>&, int, cudaStream_t);           \
    template cudaError_t launch_bounds_nodes<R>(const LanczosState<R>&, double*, int, double, double, \
                                                double, cudaStream_t);
CIQ_INSTANTIATE(float)
CIQ_INSTANTIATE(double)
#undef CIQ_INSTANTIATE

}  // namespace ciq
