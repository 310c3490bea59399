// Tensor-core (tcgen05) on-the-fly kernel MVM: interface.
#pragma once

#include "kernels.cuh"

namespace ciq {

// Rows of K per CTA (the MMA M) and columns of K per pipeline step.
constexpr int kTcBM = 128;
constexpr int kTcBN = 64;
// Bytes of one row of the augmented, split point operand: 3 chunks x 16
// 16-bit elements (x scaled and centred, the half squared norm, 1; hi/lo).
constexpr int kTcRowBytes = 96;

// Device buffers of the tensor-core MVM (inside the solve workspace).
struct TcPoints {
    uint8_t* ua = nullptr;     // points as the M operand of S = U V^T   [Npad/8][3][2][8][8] 16-bit
    uint8_t* ub = nullptr;     // points as the N operand                 same layout
    uint8_t* vblk = nullptr;   // V split hi/lo, per 64-row tile          [Npad/64][2][TP/8][8][8][8]
                               // (TF32: V rounded to TF32, per 64-row tile [Npad/64][TP/8][16][8][4])
    float* vscale = nullptr;   // power-of-two scale per column of V      [TP]
    double* mean = nullptr;    // centre of the points                    [16]
    int* err = nullptr;        // set to 1 if a bounded wait gave up
    float* part = nullptr;     // per-CTA column sums, rounded to float   [row tile][split][TP][128]
    int nsplit = 1;            // CTAs per row tile, each over a contiguous range of K's columns
    int inject = 0;            // testing only: CTA 0 skips its first point copy (its waits run out)
    int narrow = 0;            // 1: at most 8 augmented features (d <= 6), so only the first K-core
                               // of every chunk is non-zero and S takes two MMAs instead of three
    int64_t Npad = 0;
    int TP = 0;                // T rounded up to whole launch groups (32, 64 or k x 128)
    int half = 0;              // 1: FP16 operands; 0: BF16
    int tf32 = 0;              // 1: the product P V on TF32 operands (no split; points still FP16 split)
};

bool tc_supported(int precision, int d);
int tc_padded_t(int T);
int tc_group_t(int T);
int64_t tc_row_tiles(int64_t Npad);
// max_split caps the CTAs per row tile (batches, whose many problems fill the
// GPU already, use 1).
size_t tc_points_bytes(int64_t Npad, int T, int max_split = 8);
TcPoints tc_points_layout(char* base, int64_t Npad, int T, int precision, int max_split, int d);
// Centre/scale/augment/split the points (Xp: Npad x dp, already divided by
// the lengthscale) into ua/ub; clears the error flag.
cudaError_t launch_tc_prepare(const TcPoints& p, const float* Xp, int64_t N, int dp, int d, int kt,
                              cudaStream_t st);
// Split V into vblk (unit_columns: every column has norm 1, so one fixed
// power-of-two scale is used; otherwise per-column scales from the norms)
// and run the tensor-core MVM with the epilogue of `a`.
// unit_columns: V's columns have norm 1 (one power-of-two scale for all);
// scale_ready: that scale is already in p.vscale (the V-scale launch is skipped).
cudaError_t launch_mvm_tc(const TcPoints& p, const MvmArgs<float>& a, bool unit_columns, cudaStream_t st,
                          bool scale_ready = false);

// Stored K on tensor cores: O = K V with K (Npad x Npad floats, row pitch ldk,
// ldk % 4 == 0, 16-byte aligned, padded rows and columns 0) streamed by TMA,
// scaled by kscale (a power of two from stored_tc_scale(max_i K_ii), which
// bounds |K_ij| for a positive semidefinite K) and split into FP16 (p.half)
// or BF16 parts, V split as for launch_mvm_tc; p from tc_points_layout (the
// points are not used; p.err must be clear).  The epilogue of `a`, its noise
// term ignored (the stored matrix holds sigma^2).
float stored_tc_scale(double max_diag);
cudaError_t launch_stored_diag_max(const float* Kmat, int64_t ldk, int64_t N, float* out, cudaStream_t st);
cudaError_t launch_stored_mvm_tc(const float* Kmat, int64_t ldk, const TcPoints& p, const MvmArgs<float>& a,
                                 float kscale, bool unit_columns, cudaStream_t st, bool scale_ready = false);

}  // namespace ciq
