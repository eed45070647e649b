// Steering (Sec. 2.2, Eq. (10)): wavelet coefficients at arbitrary
// orientations gamma_t from the N sampled ones,
//   out[j][t][b][a] = sum_{g<N} z(gamma_t - gamma_g) W[j][g][b][a],
//   z(x) = (1/N) sum_{n in S_N} e^{i n x},  gamma_g = pi g / N.
// One pass over W: each thread reads the N samples of a (b, a) point of one
// scale once (coalesced along a) and writes its ngamma outputs; the weights
// z(gamma_t - gamma_g) arrive as a kernel parameter.  HBM-bound.
#include "internal.h"
#include "steer.h"

namespace s2dw {

// 16-byte vectors of T (4 floats or 2 doubles)
template <typename T> struct Vec16;
template <> struct Vec16<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec16<double> { using type = double2; static constexpr int n = 2; };

template <typename T>
__device__ __forceinline__ void vaxpy(typename Vec16<T>::type& s, T w, const typename Vec16<T>::type& x);
template <>
__device__ __forceinline__ void vaxpy<float>(float4& s, float w, const float4& x) {
  s.x = fma(w, x.x, s.x); s.y = fma(w, x.y, s.y); s.z = fma(w, x.z, s.z); s.w = fma(w, x.w, s.w);
}
template <>
__device__ __forceinline__ void vaxpy<double>(double2& s, double w, const double2& x) {
  s.x = fma(w, x.x, s.x); s.y = fma(w, x.y, s.y);
}

// VEC: per_scale is a multiple of the vector width (16-byte aligned rows of
// every (j, g) plane), so a thread moves 16 bytes per load and store.
template <typename T, bool VEC>
__global__ void __launch_bounds__(256) k_steer(const T* __restrict__ W, T* __restrict__ out, SteerWeights sw,
                                               int N, int ngamma, int64_t per_scale) {
  __shared__ T wt[kSteerMaxGamma][kSteerMaxN];
  // every entry: the scalar path below multiplies the unused ones (g >= N) by zero
  for (int i = threadIdx.x; i < kSteerMaxGamma * kSteerMaxN; i += blockDim.x) {
    const int t = i / kSteerMaxN, g = i % kSteerMaxN;
    wt[t][g] = (t < ngamma && g < N) ? (T)sw.w[t][g] : T(0);
  }
  __syncthreads();
  const int j = blockIdx.y;
  const T* __restrict__ Wj = W + (size_t)j * N * per_scale;
  T* __restrict__ Oj = out + (size_t)j * ngamma * per_scale;
  if constexpr (VEC) {
    using V = typename Vec16<T>::type;
    constexpr int VN = Vec16<T>::n;
    const int64_t nv = per_scale / VN;
    const V* __restrict__ Wv = reinterpret_cast<const V*>(Wj);
    V* __restrict__ Ov = reinterpret_cast<V*>(Oj);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
      V x[kSteerMaxN];
#pragma unroll
      for (int g = 0; g < kSteerMaxN; ++g)
        if (g < N) x[g] = __ldg(Wv + (size_t)g * nv + i);
      for (int t = 0; t < ngamma; ++t) {
        V s = {};
#pragma unroll
        for (int g = 0; g < kSteerMaxN; ++g)
          if (g < N) vaxpy<T>(s, wt[t][g], x[g]);
        Ov[(size_t)t * nv + i] = s;
      }
    }
  } else {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < per_scale;
         i += (int64_t)gridDim.x * blockDim.x) {
      T x[kSteerMaxN];
#pragma unroll
      for (int g = 0; g < kSteerMaxN; ++g) x[g] = g < N ? __ldg(Wj + (size_t)g * per_scale + i) : T(0);
      for (int t = 0; t < ngamma; ++t) {
        T s = 0;
#pragma unroll
        for (int g = 0; g < kSteerMaxN; ++g) s = fma(wt[t][g], x[g], s);
        Oj[(size_t)t * per_scale + i] = s;
      }
    }
  }
}

template <typename T>
cudaError_t launch_steer(const void* W, void* out, const SteerWeights& sw, int nscale, int N, int ngamma,
                         int64_t per_scale, cudaStream_t st) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const bool vec = per_scale % Vec16<T>::n == 0 && reinterpret_cast<uintptr_t>(W) % 16 == 0 &&
                   reinterpret_cast<uintptr_t>(out) % 16 == 0;
  const int64_t items = vec ? per_scale / Vec16<T>::n : per_scale;
  const int64_t want = (items + 255) / 256;
  const int bx = (int)std::min<int64_t>(want, (int64_t)sms * 8 / std::max(1, nscale) + 1);
  dim3 grid(bx, nscale);
  if (vec)
    k_steer<T, true><<<grid, 256, 0, st>>>(reinterpret_cast<const T*>(W), reinterpret_cast<T*>(out), sw, N,
                                           ngamma, per_scale);
  else
    k_steer<T, false><<<grid, 256, 0, st>>>(reinterpret_cast<const T*>(W), reinterpret_cast<T*>(out), sw, N,
                                            ngamma, per_scale);
  return cudaGetLastError();
}

template cudaError_t launch_steer<float>(const void*, void*, const SteerWeights&, int, int, int, int64_t,
                                         cudaStream_t);
template cudaError_t launch_steer<double>(const void*, void*, const SteerWeights&, int, int, int, int64_t,
                                          cudaStream_t);

}  // namespace s2dw
