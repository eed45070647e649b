// Block-level power-of-two complex FFT in shared memory (one CTA, all threads).
//
// fft_dif: in-place decimation in frequency, natural-order input ->
//          bit-reversed output, forward sign e^{-2 pi i jk/M}.
// fft_dit_inv: in-place decimation in time, bit-reversed input -> natural
//          output, sign e^{+2 pi i jk/M}, unnormalised (the result is M times
//          the inverse DFT).
// A convolution therefore needs no permutation: dif(x) .* (dif(h)/M), then
// dit_inv.  Radix-4 stages (two radix-2 stages fused, so the output order is
// plain bit reversal) plus one radix-2 stage when log2(M) is odd.
// tw[k] = e^{-2 pi i k/M}, k < M, in the working precision.
#pragma once

#include "common.cuh"

namespace s2dw {

template <typename T>
__device__ __forceinline__ void fft_dif(cx<T>* x, int logM, const cx<T>* __restrict__ tw) {
  const int M = 1 << logM;
  int span = M;
  int lg = logM;
  while (lg >= 2) {
    const int q = span >> 2;
    const int stride = M / span;
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int base = ((b - j) << 2) + j;
      cx<T> a0 = x[base], a1 = x[base + q], a2 = x[base + 2 * q], a3 = x[base + 3 * q];
      cx<T> s02 = cadd<T>(a0, a2), d02 = csub<T>(a0, a2);
      cx<T> s13 = cadd<T>(a1, a3), d13 = csub<T>(a1, a3);
      cx<T> y0 = cadd<T>(s02, s13);
      cx<T> y2 = csub<T>(s02, s13);
      cx<T> y1 = mkc<T>(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
      cx<T> y3 = mkc<T>(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
      const int t1 = j * stride;
      x[base] = y0;
      if (j == 0) {
        x[base + q] = y2;
        x[base + 2 * q] = y1;
        x[base + 3 * q] = y3;
      } else {
        x[base + q] = cmul<T>(y2, tw[2 * t1]);
        x[base + 2 * q] = cmul<T>(y1, tw[t1]);
        x[base + 3 * q] = cmul<T>(y3, tw[3 * t1]);
      }
    }
    __syncthreads();
    span >>= 2;
    lg -= 2;
  }
  if (lg == 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      cx<T> a = x[2 * b], c = x[2 * b + 1];
      x[2 * b] = cadd<T>(a, c);
      x[2 * b + 1] = csub<T>(a, c);
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ void fft_dit_inv(cx<T>* x, int logM, const cx<T>* __restrict__ tw) {
  const int M = 1 << logM;
  int span;
  if (logM & 1) {
    for (int b = threadIdx.x; b < (M >> 1); b += blockDim.x) {
      cx<T> a = x[2 * b], c = x[2 * b + 1];
      x[2 * b] = cadd<T>(a, c);
      x[2 * b + 1] = csub<T>(a, c);
    }
    __syncthreads();
    span = 8;
  } else {
    span = 4;
  }
  for (; span <= M; span <<= 2) {
    const int q = span >> 2;
    const int stride = M / span;
    for (int b = threadIdx.x; b < (M >> 2); b += blockDim.x) {
      const int j = b & (q - 1);
      const int base = ((b - j) << 2) + j;
      cx<T> y0 = x[base], p1 = x[base + q], p2 = x[base + 2 * q], p3 = x[base + 3 * q];
      cx<T> y2, y1, y3;
      if (j == 0) {
        y2 = p1;
        y1 = p2;
        y3 = p3;
      } else {
        const int t1 = j * stride;
        y2 = cmulc<T>(p1, tw[2 * t1]);
        y1 = cmulc<T>(p2, tw[t1]);
        y3 = cmulc<T>(p3, tw[3 * t1]);
      }
      cx<T> S = cadd<T>(y0, y2), D = csub<T>(y0, y2), E = cadd<T>(y1, y3);
      cx<T> dd = csub<T>(y3, y1);
      cx<T> F = mkc<T>(dd.y, -dd.x);  // -i (y3 - y1)
      x[base] = cadd<T>(S, E);
      x[base + q] = cadd<T>(D, F);
      x[base + 2 * q] = csub<T>(S, E);
      x[base + 3 * q] = csub<T>(D, F);
    }
    __syncthreads();
  }
}

}  // namespace s2dw
