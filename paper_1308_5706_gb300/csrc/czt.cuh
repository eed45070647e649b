// Chirp-z kernels for the beta and alpha sums of the analysis (Sec. 3.2,
// Eqs. (29)-(30)) and the alpha and beta quadratures of the synthesis
// (Sec. 3.3, Eqs. (37) and (40)).
//
// Every sum has the form X_d = sum_s x_s e^{i 2 theta s d} over a contiguous
// range of s and d, evaluated as
//   X_d = e^{i theta d^2} sum_s (x_s e^{i theta s^2}) e^{-i theta (d-s)^2}
// with a circular convolution of power-of-two length M >= 4L-2 (the radix-16
// engine of fft16.cuh, one CTA per transform): inputs sit at
// s mod M, outputs are read at d mod M, and the kernel h_u is stored at
// u mod M for the whole u-range any scale can need, so one spectrum per
// plan serves every scale.  theta = pi/(4L) for beta (beta_b = theta(2b+1))
// and pi/(2L-1) for alpha (alpha_a = 2 theta a).
//
// Layouts (measured choices): analysis Y_g[m][m'] (m' fastest: the beta
// step reads contiguous columns) and X_g[b][m] (m fastest: alpha reads rows);
// synthesis V_g[b][m] (alpha writes rows) and Vhat_g[m'][m] (the contraction
// prologue reads it coalesced), so the synthesis beta step reads and writes
// strided columns.
// beta, analysis:  X_g[b][m] = sum_{|m'|<Lj} Yhat_{m'} e^{i m' beta_b},
//   Yhat_{-m'} = sigma_m Yhat_{m'}, sigma_m = (-1)^{m+N-1}   (one column / CTA)
// alpha, analysis: W[a] = sum_{|m|<Lj} X_m e^{i m alpha_a}, X_{-m} = conj(X_m);
//   two real rows per complex transform                      (one pair / CTA)
// alpha, synthesis: V_m = 2pi/(2L-1) sum_a W_a e^{-i m alpha_a}, m < Lj
// beta, synthesis: T_{m'} = sum_b q_b V_b e^{-i m' beta_b},
//   Vhat_{m'} = T_{m'} + sigma_m T_{-m'} (m' > 0), Vhat_0 = T_0  (Eq. (40)
//   folded over +-m' so that every integrand is a cosine series).
#pragma once

#include "fft16.cuh"
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
__global__ void __launch_bounds__(256) k_czt_beta_ana(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM;
  const int g = item / Lj, m = item % Lj;
  const T sigma = ((m + sg.N - 1) & 1) ? T(-1) : T(1);
  const cx<T>* __restrict__ Y = sg.buf_in + ((size_t)g * Lj + m) * Lj;  // Y_g[m][.], m' fastest
  const cx<T>* __restrict__ pre = sg.pre + (L - 1);
  auto in = [&](int v) -> cx<T> {
    int mp;
    if (v < Lj) mp = v;
    else if (v > M - Lj) mp = v - M;
    else return mkc<T>(0, 0);
    cx<T> y = Y[mp < 0 ? -mp : mp];
    if (mp < 0) y = cscale<T>(y, sigma);
    return cmul<T>(y, __ldg(pre + mp));
  };
  cx<T>* __restrict__ X = sg.buf_out + (size_t)g * 2 * L * Lj + m;
  auto out = [&](int v, cx<T> val) {
    if (v < 2 * L) X[(size_t)v * Lj] = cmul<T>(val, __ldg(sg.post + v));
  };
  fft_convolve<T, false>(A, sg.logM, sg.H, sg.tw, in, out);
}

template <typename T>
__global__ void __launch_bounds__(256) k_czt_alpha_ana(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM, n = 2 * L - 1;
  const int r1 = 2 * item;  // rows r1, r1 + 1 of the [N * 2L] row space
  const cx<T>* __restrict__ X1 = sg.buf_in + (size_t)r1 * Lj;
  const cx<T>* __restrict__ X2 = X1 + Lj;
  auto in = [&](int v) -> cx<T> {
    int mm;
    bool neg;
    if (v < Lj) {
      mm = v;
      neg = false;
    } else if (v > M - Lj) {
      mm = M - v;
      neg = true;
    } else {
      return mkc<T>(0, 0);
    }
    const cx<T> x1 = X1[mm], x2 = X2[mm];
    const cx<T> z = neg ? mkc<T>(x1.x + x2.y, x2.x - x1.y)    // conj(X1) + i conj(X2)
                        : mkc<T>(x1.x - x2.y, x1.y + x2.x);   // X1 + i X2
    return cmul<T>(z, __ldg(sg.pre + mm));
  };
  T* __restrict__ Wb = reinterpret_cast<T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff;
  T* __restrict__ W1 = Wb + (size_t)r1 * n;
  T* __restrict__ W2 = W1 + n;
  auto out = [&](int v, cx<T> val) {
    if (v < n) {
      const cx<T> w = cmul<T>(val, __ldg(sg.post + v));
      W1[v] = w.x;
      W2[v] = w.y;
    }
  };
  fft_convolve<T, false>(A, sg.logM, sg.H, sg.tw, in, out);
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
  auto in = [&](int v) -> cx<T> {
    if (v >= n) return mkc<T>(0, 0);
    return cmulc<T>(mkc<T>(W1[v], W2[v]), __ldg(sg.pre + v));
  };
  auto none = [](int, cx<T>) {};
  fft_convolve<T, true>(A, sg.logM, sg.H, sg.tw, in, none);
  cx<T>* __restrict__ V1 = sg.buf_out + (size_t)r1 * Lj;  // V_g[b][m] rows, m fastest
  cx<T>* __restrict__ V2 = V1 + Lj;
  const T h = sg.scale * T(0.5);
  for (int mm = threadIdx.x; mm < Lj; mm += blockDim.x) {
    const cx<T> ch = __ldg(sg.post + mm);
    const cx<T> zp = cmulc<T>(A[fpad(mm)], ch);
    const cx<T> zm = cmulc<T>(A[fpad((M - mm) & (M - 1))], ch);
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
  const cx<T>* __restrict__ V = sg.buf_in + (size_t)g * 2 * L * Lj + m;  // column m of V_g[b][m]
  auto in = [&](int v) -> cx<T> {
    if (v >= 2 * L) return mkc<T>(0, 0);
    return cmul<T>(V[(size_t)v * Lj], __ldg(sg.pre + v));
  };
  auto none = [](int, cx<T>) {};
  fft_convolve<T, true>(A, sg.logM, sg.H, sg.tw, in, none);
  cx<T>* __restrict__ Vh = sg.buf_out + (size_t)g * Lj * Lj + m;  // column m of Vhat_g[m'][m]
  for (int mp = threadIdx.x; mp < Lj; mp += blockDim.x) {
    const cx<T> tp = cmul<T>(A[fpad(mp)], __ldg(sg.post + L - 1 + mp));
    cx<T> o = tp;
    if (mp > 0) {
      const cx<T> tm = cmul<T>(A[fpad(M - mp)], __ldg(sg.post + L - 1 - mp));
      o = mkc<T>(tp.x + sigma * tm.x, tp.y + sigma * tm.y);
    }
    Vh[(size_t)mp * Lj] = o;
  }
}

template <typename T>
void launch_czt_impl(int kind, const CztSeg<T>* segs, int nseg, int total_items, int maxlogM,
                     const CallPtrs& ptrs, cudaStream_t st) {
  if (total_items <= 0) return;
  const size_t smem = sizeof(cx<T>) * (size_t)fft_smem_elems(1 << maxlogM);
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
  const int smem = (int)(sizeof(cx<T>) * (size_t)fft_smem_elems(1 << maxlogM));
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
