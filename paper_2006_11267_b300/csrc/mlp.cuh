// Learned spectral-bound predictor (see mlp.cu): sizes, parameter layout and launchers.
#pragma once

#include "common.cuh"

namespace ciq {

constexpr int kMlpIn = CIQ_MLP_INPUTS;
constexpr int kMlpHid = 64;
constexpr int kMlpOut = CIQ_MLP_OUTPUTS;
constexpr int kMlpOffW1 = 2 * kMlpIn + 2 * kMlpOut;
constexpr int kMlpOffB1 = kMlpOffW1 + kMlpIn * kMlpHid;
constexpr int kMlpOffW2 = kMlpOffB1 + kMlpHid;
constexpr int kMlpOffB2 = kMlpOffW2 + kMlpHid * kMlpHid;
constexpr int kMlpOffW3 = kMlpOffB2 + kMlpHid;
constexpr int kMlpOffB3 = kMlpOffW3 + kMlpHid * kMlpOut;
constexpr int kMlpParams = kMlpOffB3 + kMlpOut;
static_assert(kMlpParams == CIQ_MLP_PARAMS, "parameter count of the header");

cudaError_t launch_mlp_features(const ciq_problem* probs_dev, int P, float* F, cudaStream_t st);
cudaError_t launch_mlp_normaliser(const float* F, const float* Y, int n, float* theta, cudaStream_t st);
cudaError_t launch_mlp_init(float* theta, uint64_t seed, cudaStream_t st);
cudaError_t launch_mlp_loss_grad(const float* theta, const float* F, const float* Y, int n, double* loss,
                                 double* grad, cudaStream_t st);
cudaError_t launch_mlp_train(float* theta, float* adam, const float* F, const float* Y, int n, int steps, int batch,
                             float lr, uint64_t seed, int first_step, float* losses, cudaStream_t st);
cudaError_t launch_mlp_predict(const float* theta, const float* F, int n, float* out, int bf16, cudaStream_t st);

}  // namespace ciq
