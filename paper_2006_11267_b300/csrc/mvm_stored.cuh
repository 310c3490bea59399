// Stored-K kernel MVM: interface.
#pragma once

#include "kernels.cuh"

namespace ciq {

// Rows of partial sums the stored MVM writes for T columns.
int64_t stored_row_tiles(int64_t Npad, int T);
// K = K_XX + sigma^2 I from points Xp (Npad x dp, divided by the lengthscale)
// into rows [0, Npad) and columns [0, ncols) of Kmat; 0 outside [0, N)^2.
cudaError_t launch_kernel_matrix(const float* Xp, int64_t N, int64_t Npad, int dp, int kt, float s,
                                 float noise, float* Kmat, int64_t ldk, int64_t ncols, cudaStream_t st);
// O = Kmat V with the epilogue of `a` (its noise term is ignored: the stored
// matrix holds sigma^2).  Kmat: Npad rows, ldk >= Npad, ldk % 4 == 0.
cudaError_t launch_stored_mvm(const float* Kmat, int64_t ldk, const MvmArgs<float>& a, cudaStream_t st);

}  // namespace ciq
