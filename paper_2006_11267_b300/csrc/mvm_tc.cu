// Tensor-core (tcgen05) on-the-fly kernel MVM.
#include "mvm_tc.cuh"

namespace ciq {

bool tc_supported(int precision, int d) { (void)precision; (void)d; return false; }
int64_t tc_row_tiles(int64_t Npad) { return Npad / 128; }
size_t tc_points_bytes(int64_t Npad, int d) { (void)Npad; (void)d; return 0; }
TcPoints tc_points_layout(char* base, int64_t Npad, int d) { (void)Npad; (void)d; TcPoints p; p.a = base; return p; }
cudaError_t launch_tc_prepare(const TcPoints&, const float*, int64_t, int, int, int, cudaStream_t) {
    return cudaErrorNotSupported;
}
cudaError_t launch_mvm_tc(const TcPoints&, const MvmArgs<float>&, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

}  // namespace ciq
