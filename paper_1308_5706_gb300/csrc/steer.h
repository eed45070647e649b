// Steering kernel interface (Eq. (10)); weights are computed on the host.
#pragma once

#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

namespace s2dw {

constexpr int kSteerMaxGamma = 32;
constexpr int kSteerMaxN = 8;

// z(gamma_t - gamma_g), float64, t < ngamma, g < N (kernel parameter, 2 KB)
struct SteerWeights {
  double w[kSteerMaxGamma][kSteerMaxN];
};

template <typename T>
cudaError_t launch_steer(const void* W, void* out, const SteerWeights& sw, int nscale, int N, int ngamma,
                         int64_t per_scale, cudaStream_t st);

}  // namespace s2dw
