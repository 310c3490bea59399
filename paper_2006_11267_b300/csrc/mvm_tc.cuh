// Tensor-core (tcgen05) on-the-fly kernel MVM: interface.
#pragma once

#include "kernels.cuh"

namespace ciq {

// Device copies of the points in the operand formats of the tensor-core MVM.
struct TcPoints {
    void* a = nullptr;        // augmented, split operand rows (format depends on precision)
    size_t bytes = 0;
};

bool tc_supported(int precision, int d);
int64_t tc_row_tiles(int64_t Npad);
size_t tc_points_bytes(int64_t Npad, int d);
TcPoints tc_points_layout(char* base, int64_t Npad, int d);
cudaError_t launch_tc_prepare(const TcPoints& p, const float* Xp, int64_t Npad, int dp, int d,
                              int precision, cudaStream_t st);
cudaError_t launch_mvm_tc(const TcPoints& p, const MvmArgs<float>& a, int precision, cudaStream_t st);

}  // namespace ciq
