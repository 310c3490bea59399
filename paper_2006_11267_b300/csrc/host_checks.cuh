// Host-side argument checks shared by the C entry points of libciq.
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "ciq.h"

namespace ciq {

// A kernel description the library accepts: a known type, lengthscale and
// outputscale finite and > 0, noise (sigma^2) finite and >= 0.
inline bool valid_kernel(const ciq_kernel* k) {
    return k && (k->type == CIQ_RBF || k->type == CIQ_MATERN52) && k->lengthscale > 0.0 &&
           std::isfinite(k->lengthscale) && k->outputscale > 0.0 && std::isfinite(k->outputscale) &&
           k->noise >= 0.0 && std::isfinite(k->noise);
}

// True when kernels can dereference p directly (device or managed memory).
inline bool device_accessible(const void* p) {
    if (p == nullptr) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Point dimension padded to the 4-float rows of the scaled point array.
inline int dim_pad(int d) { return (d + 3) / 4 * 4; }

}  // namespace ciq
