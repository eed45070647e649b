// Chirp-z kernels for the beta and alpha sums of the analysis (Sec. 3.2,
// Eqs. (29)-(30)) and the alpha and beta quadratures of the synthesis
// (Sec. 3.3, Eqs. (37) and (40)).
//
// Every sum has the form X_d = sum_s x_s e^{i 2 theta s d} over a contiguous
// range of s and d, evaluated as
//   X_d = e^{i theta d^2} sum_s (x_s e^{i theta s^2}) e^{-i theta (d-s)^2}
// with a circular convolution of power-of-two length M >= 4L-2: inputs sit at
// s mod M, outputs are read at d mod M, and the kernel h_u is stored at
// u mod M for the whole u-range any scale can need, so one spectrum per
// plan serves every scale.  theta = pi/(4L) for beta (beta_b = theta(2b+1))
// and pi/(2L-1) for alpha (alpha_a = 2 theta a).
//
// beta, analysis:  X_g[b][m] = sum_{|m'|<Lj} Yhat_{m'} e^{i m' beta_b},
//   Yhat_{-m'} = sigma_m Yhat_{m'}, sigma_m = (-1)^{m+N-1}   (one column / CTA)
// alpha, analysis: W[a] = sum_{|m|<Lj} X_m e^{i m alpha_a}, X_{-m} = conj(X_m);
//   two real rows per complex transform                      (one pair / CTA)
// alpha, synthesis: V_m = 2pi/(2L-1) sum_a W_a e^{-i m alpha_a}, m < Lj
// beta, synthesis: T_{m'} = sum_b q_b V_b e^{-i m' beta_b},
//   Vhat_{m'} = T_{m'} + sigma_m T_{-m'} (m' > 0), Vhat_0 = T_0  (Eq. (40)
//   folded over +-m' so that every integrand is a cosine series).
#pragma once

#include "fft.cuh"
#include "internal.h"

namespace s2dw {

template <typename T>
__device__ __forceinline__ int czt_find_seg(const CztSeg<T>* segs, int nseg) {
  int lo = 0, hi = nseg - 1;
  const int b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

template <typename T>
__device__ __forceinline__ void czt_convolve(cx<T>* A, int logM, const cx<T>* __restrict__ H,
                                             const cx<T>* __restrict__ tw) {
  __syncthreads();
  fft_dif<T>(A, logM, tw);
  const int M = 1 << logM;
  for (int v = threadIdx.x; v < M; v += blockDim.x) A[v] = cmul<T>(A[v], __ldg(H + v));
  __syncthreads();
  fft_dit_inv<T>(A, logM, tw);
}

template <typename T>
__global__ void __launch_bounds__(256) k_czt_beta_ana(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM;
  const int g = item / Lj, m = item % Lj;
  const T sigma = ((m + sg.N - 1) & 1) ? T(-1) : T(1);
  for (int v = threadIdx.x; v < M; v += blockDim.x) A[v] = mkc<T>(0, 0);
  __syncthreads();
  const cx<T>* __restrict__ Y = sg.buf_in + (size_t)g * Lj * Lj + m;
  for (int mp = threadIdx.x; mp < Lj; mp += blockDim.x) {
    const cx<T> y = Y[(size_t)mp * Lj];
    A[mp] = cmul<T>(y, __ldg(sg.pre + mp + L - 1));
    if (mp > 0) A[M - mp] = cmul<T>(cscale<T>(y, sigma), __ldg(sg.pre + L - 1 - mp));
  }
  czt_convolve<T>(A, sg.logM, sg.H, sg.tw);
  cx<T>* __restrict__ X = sg.buf_out + (size_t)g * 2 * L * Lj + m;
  for (int b = threadIdx.x; b < 2 * L; b += blockDim.x) X[(size_t)b * Lj] = cmul<T>(A[b], __ldg(sg.post + b));
}

template <typename T>
__global__ void __launch_bounds__(256) k_czt_alpha_ana(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM, n = 2 * L - 1;
  const int r1 = 2 * item;  // rows r1, r1 + 1 of the [N * 2L] row space
  for (int v = threadIdx.x; v < M; v += blockDim.x) A[v] = mkc<T>(0, 0);
  __syncthreads();
  const cx<T>* __restrict__ X1 = sg.buf_in + (size_t)r1 * Lj;
  const cx<T>* __restrict__ X2 = X1 + Lj;
  for (int mm = threadIdx.x; mm < Lj; mm += blockDim.x) {
    const cx<T> x1 = X1[mm], x2 = X2[mm];
    const cx<T> ch = __ldg(sg.pre + mm);
    A[mm] = cmul<T>(mkc<T>(x1.x - x2.y, x1.y + x2.x), ch);              // X1 + i X2
    if (mm > 0) A[M - mm] = cmul<T>(mkc<T>(x1.x + x2.y, x2.x - x1.y), ch);  // conj(X1) + i conj(X2)
  }
  czt_convolve<T>(A, sg.logM, sg.H, sg.tw);
  T* __restrict__ Wb = reinterpret_cast<T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff;
  T* __restrict__ W1 = Wb + (size_t)r1 * n;
  T* __restrict__ W2 = W1 + n;
  for (int a = threadIdx.x; a < n; a += blockDim.x) {
    const cx<T> v = cmul<T>(A[a], __ldg(sg.post + a));
    W1[a] = v.x;
    W2[a] = v.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_czt_alpha_syn(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM, n = 2 * L - 1;
  const int r1 = 2 * item;
  const T* __restrict__ Wb = reinterpret_cast<const T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff;
  const T* __restrict__ W1 = Wb + (size_t)r1 * n;
  const T* __restrict__ W2 = W1 + n;
  for (int v = threadIdx.x; v < M; v += blockDim.x) {
    cx<T> z = mkc<T>(0, 0);
    if (v < n) z = cmulc<T>(mkc<T>(W1[v], W2[v]), __ldg(sg.pre + v));
    A[v] = z;
  }
  czt_convolve<T>(A, sg.logM, sg.H, sg.tw);
  cx<T>* __restrict__ V1 = sg.buf_out + (size_t)r1 * Lj;
  cx<T>* __restrict__ V2 = V1 + Lj;
  const T h = sg.scale * T(0.5);
  for (int mm = threadIdx.x; mm < Lj; mm += blockDim.x) {
    const cx<T> ch = __ldg(sg.post + mm);
    const cx<T> zp = cmulc<T>(A[mm], ch);
    const cx<T> zm = cmulc<T>(A[(M - mm) & (M - 1)], ch);
    // V1 = (Zp + conj(Zm))/2, V2 = (Zp - conj(Zm))/(2i)
    V1[mm] = mkc<T>((zp.x + zm.x) * h, (zp.y - zm.y) * h);
    V2[mm] = mkc<T>((zp.y + zm.y) * h, (zm.x - zp.x) * h);
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_czt_beta_syn(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM;
  const int g = item / Lj, m = item % Lj;
  const T sigma = ((m + sg.N - 1) & 1) ? T(-1) : T(1);
  const cx<T>* __restrict__ V = sg.buf_in + (size_t)g * 2 * L * Lj + m;
  for (int v = threadIdx.x; v < M; v += blockDim.x) {
    cx<T> z = mkc<T>(0, 0);
    if (v < 2 * L) z = cmul<T>(V[(size_t)v * Lj], __ldg(sg.pre + v));
    A[v] = z;
  }
  czt_convolve<T>(A, sg.logM, sg.H, sg.tw);
  cx<T>* __restrict__ Vh = sg.buf_out + (size_t)g * Lj * Lj + m;
  for (int mp = threadIdx.x; mp < Lj; mp += blockDim.x) {
    const cx<T> tp = cmul<T>(A[mp], __ldg(sg.post + L - 1 + mp));
    cx<T> out = tp;
    if (mp > 0) {
      const cx<T> tm = cmul<T>(A[M - mp], __ldg(sg.post + L - 1 - mp));
      out = mkc<T>(tp.x + sigma * tm.x, tp.y + sigma * tm.y);
    }
    Vh[(size_t)mp * Lj] = out;
  }
}

template <typename T>
void launch_czt_impl(int kind, const CztSeg<T>* segs, int nseg, int total_items, int maxlogM,
                     const CallPtrs& ptrs, cudaStream_t st) {
  if (total_items <= 0) return;
  const size_t smem = sizeof(cx<T>) << maxlogM;
  dim3 grid(total_items), block(256);
  switch (kind) {
    case CZT_BETA_ANA: k_czt_beta_ana<T><<<grid, block, smem, st>>>(segs, nseg); break;
    case CZT_ALPHA_ANA: k_czt_alpha_ana<T><<<grid, block, smem, st>>>(segs, nseg, ptrs); break;
    case CZT_ALPHA_SYN: k_czt_alpha_syn<T><<<grid, block, smem, st>>>(segs, nseg, ptrs); break;
    case CZT_BETA_SYN: k_czt_beta_syn<T><<<grid, block, smem, st>>>(segs, nseg); break;
    default: break;
  }
}

template <typename T>
cudaError_t czt_set_smem(int maxlogM) {
  const int smem = (int)(sizeof(cx<T>) << maxlogM);
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_czt_beta_ana<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_czt_alpha_ana<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_czt_alpha_syn<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_czt_beta_syn<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace s2dw
