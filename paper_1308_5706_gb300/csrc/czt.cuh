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

#include <algorithm>
#include <mutex>
#include <vector>

#include "fft16.cuh"
#include "internal.h"

namespace s2dw {

template <typename T>
__device__ __forceinline__ int czt_find_seg(const CztSeg<T>* segs, int nseg, int b = -1) {
  int lo = 0, hi = nseg - 1;
  if (b < 0) b = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (segs[mid].start <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// NT adjacent columns m0.. per CTA (the segment's P: FP32 two up to M = 2^12,
// so that each output row b gets both columns in one 16-byte store, one at
// M = 2^13 so that a CTA's buffers stay at 69.6 KB).  M >= 4L: the inputs
// (|m'| < L_j <= M/4) sit in the first and last quarter of the period, the
// outputs b < nb <= 2L in the first half.
// buffer elements of the chirp-z beta kernels for segments up to length 2^maxlogM
inline size_t beta_czt_smem_elems(int maxlogM, bool fp64) {
  size_t e = 0;
  for (int lm = 5; lm <= maxlogM; ++lm)
    e = std::max(e, (size_t)beta_czt_cols(lm, fp64) * (size_t)fft_smem_elems(1 << lm));
  return e;
}

template <typename T, int NT>
__device__ __forceinline__ void czt_beta_ana_body(const CztSeg<T>& sg, cx<T>* A) {
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM, ST = fft_smem_elems(M);
  const int per_g = (Lj + NT - 1) / NT;
  const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, Lj - m0);
  const cx<T>* __restrict__ pre = sg.pre + (L - 1);
  const cx<T>* __restrict__ Y0 = sg.buf_in + ((size_t)g * Lj + m0) * Lj;  // Y_g[m0 + t][.], m' fastest
  auto pref = [&](int v) -> cx<T> {
    if (v < Lj) return ldk(pre + v);
    if (v > M - Lj) return ldk(pre + (v - M));
    return mkc<T>(0, 0);
  };
  auto in = [&](int v, int t, cx<T> c) -> cx<T> {
    if (t >= nt) return mkc<T>(0, 0);
    const cx<T>* __restrict__ Y = Y0 + (size_t)t * Lj;
    if (v < Lj) return cmul<T>(Y[v], c);
    if (v > M - Lj) {
      const T sigma = ((m0 + t + sg.N - 1) & 1) ? T(-1) : T(1);
      return cmul<T>(cscale<T>(Y[M - v], sigma), c);
    }
    return mkc<T>(0, 0);
  };
  auto nopost = [](int) -> cx<T> { return mkc<T>(0, 0); };
  auto none = [](int, int, cx<T>, cx<T>) {};
  cx<T>* __restrict__ X = sg.buf_out + (size_t)g * sg.nb * Lj + m0;
  // An odd row count N nb (MW grid) pairs the last row with row N nb of the
  // buffer (which holds 2L rows per gamma sample) in the alpha analysis: zero it.
  if (g == sg.N - 1 && ((sg.N * sg.nb) & 1) && threadIdx.x < nt) X[(size_t)sg.nb * Lj + threadIdx.x] = mkc<T>(0, 0);
  fft_convolve_n<T, NT, true, 0xF00Fu, 0x00FFu>(A, ST, sg.logM, sg.H, sg.tw, pref, in, nopost, none, []() {});
  const bool pair = NT == 2 && nt == 2 && (Lj & 1) == 0;  // 16-byte aligned column pairs
  for (int b = threadIdx.x; b < sg.nb; b += blockDim.x) {
    const cx<T> c = ldk(sg.post + b);
    cx<T>* __restrict__ xr = X + (size_t)b * Lj;
    if (pair) {
      const cx<T> y0 = cmul<T>(A[fpad(b)], c), y1 = cmul<T>(A[ST + fpad(b)], c);
      *reinterpret_cast<float4*>(xr) = make_float4(y0.x, y0.y, y1.x, y1.y);
    } else {
      for (int t = 0; t < nt; ++t) xr[t] = cmul<T>(A[t * ST + fpad(b)], c);
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_czt_beta_ana(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  if (sizeof(T) == sizeof(float) && sg.P == 2) czt_beta_ana_body<T, 2>(sg, A);
  else czt_beta_ana_body<T, 1>(sg, A);
}

// MW grid, synthesis: the beta dependence of a (g, m) column of V is a
// trigonometric polynomial of degree < L_j with V(2 pi - beta) = sigma
// V(beta), sigma = (-1)^{m+n} (d^l_mn(-beta) = (-1)^{m-n} d^l_mn(beta); all
// orders n have the parity of N-1).  Its L samples beta_b = (2b+1) pi / n and
// their reflections are the n = 2L-1 equispaced points of the torus, so
//   c_p = (1/n) sum_{b<n} V(beta_b) e^{-i p beta_b},  0 <= p < L_j
// are its Fourier coefficients exactly (c_{-p} = sigma c_p).  Chirp-z of
// length M: c_p = (1/n) e^{-i pi (p^2 + p)/n} sum_b [V_b e^{-i pi b^2/n}]
// e^{+i pi (p - b)^2/n}.  Output in the Y layout [g][m][p] that the beta
// evaluation kernels read, which then give the column on the DH grid.
template <typename T, int NT>  // NT adjacent columns per CTA (the segment's P)
__device__ __forceinline__ void beta_mw_dft_body(const CztSeg<T>& sg, cx<T>* A) {
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, n = 2 * L - 1, M = 1 << sg.logM, ST = fft_smem_elems(M);
  const int per_g = (Lj + NT - 1) / NT;
  const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, Lj - m0);
  const cx<T>* __restrict__ V = sg.buf_in + (size_t)g * sg.nb * Lj + m0;  // columns m0.. of V_g[b][m], b < L
  auto pref = [&](int v) -> cx<T> { return v < n ? ldk(sg.pre + v) : mkc<T>(0, 0); };  // e^{i pi b^2/n}
  auto in = [&](int v, int t, cx<T> c) -> cx<T> {
    if (v >= n || t >= nt) return mkc<T>(0, 0);
    const T sigma = ((m0 + t + sg.N - 1) & 1) ? T(-1) : T(1);
    // beta = pi (v = L - 1) is its own reflection: a sigma = -1 column vanishes there
    const cx<T> x = v < L ? cscale<T>(V[(size_t)v * Lj + t], (v == L - 1 && sigma < T(0)) ? T(0) : T(1))
                          : cscale<T>(V[(size_t)(n - 1 - v) * Lj + t], sigma);
    return cmulc<T>(x, c);
  };
  auto nopost = [](int) -> cx<T> { return mkc<T>(0, 0); };
  auto none = [](int, int, cx<T>, cx<T>) {};
  // inputs v < n <= M/2; outputs p < L_j <= M/4
  fft_convolve_n<T, NT, true, 0x00FFu, 0x000Fu>(A, ST, sg.logM, sg.H, sg.tw, pref, in, nopost, none, []() {});
  const T inv_n = T(1) / T(n);
  for (int t = 0; t < nt; ++t) {
    cx<T>* __restrict__ C = sg.buf_out + ((size_t)g * Lj + m0 + t) * Lj;  // c_p, p < Lj
    for (int v = threadIdx.x; v < Lj; v += blockDim.x)
      C[v] = cscale<T>(cmulc<T>(A[t * ST + fpad(v)], ldk(sg.post + (L - 1) + v)), inv_n);  // sg.post: MW chirp
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_beta_mw_dft(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  if (sizeof(T) == sizeof(float) && sg.P == 2) beta_mw_dft_body<T, 2>(sg, A);
  else beta_mw_dft_body<T, 1>(sg, A);
}

// alpha sums: item `it` is NT row pairs (rows 2(it' NT + t), +1, t < NT, it'
// the item's index in its segment).  The synthesis kernel is persistent (a
// grid of a few CTAs per SM walks the items): while a CTA computes one item,
// cp.async stages the W rows of its next item in shared memory, so the HBM
// latency of the inputs is hidden behind the FFT work.
// Shared memory: NT FFT buffers of ST = fft_smem_elems(2^maxlogM) complex,
// then (synthesis) the staging rows (2 NT rows of pitch 2^(maxlogM-1) of T).
template <typename T>
__host__ __device__ constexpr size_t alpha_czt_smem(int maxlogM, bool staging) {
  return (size_t)alpha_czt_nt(sizeof(T) == 8) *
         ((size_t)fft_smem_elems(1 << maxlogM) * sizeof(cx<T>) +
          (staging ? 2 * ((size_t)1 << (maxlogM - 1)) * sizeof(T) : 0));
}

// The analysis form is not persistent: its inputs (the X rows the beta step
// has just written) are mostly L2-resident and few, so one CTA per item with
// direct loads measured faster than staging them ahead.
// ODD: some segment may have an odd row count (MW grid); the DH grid's even
// counts compile without the guards.
// LOGM > 0 (here and in the kernels below): every segment of the launch has
// transforms of length 2^LOGM, a compile-time length; 0: any.
// ahead: CTAs resident at once; a CTA asks L2 for the X rows of the CTA
// `ahead` places later, which runs about one wave later.
template <typename T, bool ODD, int LOGM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_czt_alpha_ana(const CztSeg<T>* __restrict__ segs, int nseg, int maxlogM,
                                                          CallPtrs ptrs, int ahead) {
  constexpr int NT = alpha_czt_nt(sizeof(T) == 8);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const int ST = fft_smem_elems(1 << maxlogM);
  if (threadIdx.x == 0 && blockIdx.x + ahead < gridDim.x) {
    const CztSeg<T>& s2 = segs[czt_find_seg<T>(segs, nseg, blockIdx.x + ahead)];
    const int q0 = (blockIdx.x + ahead - s2.start) * NT, nr = min(2 * NT, s2.N * s2.nb - 2 * q0);
    if (nr > 0) prefetch_l2(s2.buf_in + (size_t)(2 * q0) * s2.Lj, (size_t)nr * s2.Lj * sizeof(cx<T>));
  }
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int logM = LOGM ? LOGM : sg.logM;
  const int Lj = sg.Lj, L = sg.L, M = 1 << logM, n = 2 * L - 1;
  const int p0 = (blockIdx.x - sg.start) * NT;
  const int rows = sg.N * sg.nb;           // rows (g, b); row pair p = rows 2p, 2p+1
  const int nt = min(NT, (ODD ? rows + 1 : rows) / 2 - p0);  // transforms present in this CTA
  const cx<T>* __restrict__ X = sg.buf_in + (size_t)(2 * p0) * Lj;
  // input position v holds m = v (v < Lj) or m = v - M (v > M - Lj)
  auto pre = [&](int v) -> cx<T> {
    if (v < Lj) return ldk(sg.pre + v);
    if (v > M - Lj) return ldk(sg.pre + (M - v));
    return mkc<T>(0, 0);
  };
  // an odd row count (MW grid) leaves the last pair one row; its partner is
  // the zero row that the beta analysis writes after the last row
  auto two = [&](int t) { return !ODD || 2 * (p0 + t) + 1 < rows; };
  auto in = [&](int v, int t, cx<T> c) -> cx<T> {
    if (t >= nt) return mkc<T>(0, 0);
    // X is read once: streaming loads keep L1 for the tables
    if (v < Lj) {
      const cx<T> x1 = __ldcs(X + (size_t)(2 * t) * Lj + v), x2 = __ldcs(X + (size_t)(2 * t + 1) * Lj + v);
      return cmul<T>(mkc<T>(x1.x - x2.y, x1.y + x2.x), c);  // X1 + i X2
    }
    if (v > M - Lj) {
      const int mm = M - v;
      const cx<T> x1 = __ldcs(X + (size_t)(2 * t) * Lj + mm), x2 = __ldcs(X + (size_t)(2 * t + 1) * Lj + mm);
      return cmul<T>(mkc<T>(x1.x + x2.y, x2.x - x1.y), c);  // conj(X1) + i conj(X2)
    }
    return mkc<T>(0, 0);
  };
  T* __restrict__ Wb = reinterpret_cast<T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff +
                       (size_t)(2 * p0) * n;
  auto post = [&](int v) -> cx<T> { return v < n ? ldk(sg.post + v) : mkc<T>(0, 0); };
  auto out = [&](int v, int t, cx<T> y, cx<T> c) {
    if (v < n && t < nt) {
      const cx<T> w = cmul<T>(y, c);
      __stcs(Wb + (size_t)(2 * t) * n + v, w.x);
      if (two(t)) __stcs(Wb + (size_t)(2 * t + 1) * n + v, w.y);
    }
  };
  // M >= 4L: the inputs (|m| < L_j <= M/4) sit in the first and last
  // quarter of the period, the n = 2L-1 outputs in the first half
  fft_convolve_n<T, NT, false, 0xF00Fu, 0x00FFu>(A, ST, logM, sg.H, sg.tw, pre, in, post, out, []() {});
}

template <typename T, int LOGM>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 3 : 2) k_czt_alpha_syn(const CztSeg<T>* __restrict__ segs, int nseg, int total,
                                                          int maxlogM, CallPtrs ptrs) {
  constexpr int NT = alpha_czt_nt(sizeof(T) == 8);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const int ST = fft_smem_elems(1 << maxlogM);
  const int P = 1 << (maxlogM - 1);  // staging pitch in elements of T (>= 2L > n)
  T* stg = reinterpret_cast<T*>(A + NT * ST);  // [2 NT][P] W rows of the next item
  auto prefetch = [&](int it) {
    if (it < total) {
      const CztSeg<T> sp = segs[czt_find_seg<T>(segs, nseg, it)];
      const int p0 = (it - sp.start) * NT, n = 2 * sp.L - 1;
      const int nr = min(2 * NT, sp.N * sp.nb - 2 * p0);  // rows of this item (the last pair may have one)
      const T* __restrict__ Wr = reinterpret_cast<const T*>(sp.is_phi ? ptrs.Wphi[sp.job] : ptrs.W[sp.job]) +
                                 sp.woff + (size_t)(2 * p0) * n;
      for (int r = 0; r < nr; ++r)
        for (int a = threadIdx.x; a < n; a += blockDim.x)
          cp_async_ca<sizeof(T)>(stg + r * P + a, Wr + (size_t)r * n + a);
      if (nr & 1)  // the missing second row of the last pair (MW grid, odd row count): zeros
        for (int a = threadIdx.x; a < n; a += blockDim.x) stg[nr * P + a] = T(0);
    }
    cp_async_commit();
  };
  int it = blockIdx.x;
  prefetch(it);
  for (; it < total; it += gridDim.x) {
    const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg, it)];
    const int logM = LOGM ? LOGM : sg.logM;
    const int Lj = sg.Lj, L = sg.L, M = 1 << logM, n = 2 * L - 1;
    const int p0 = (it - sg.start) * NT;
    const int rows = sg.N * sg.nb;
    const int nt = min(NT, (rows + 1) / 2 - p0);
    cp_async_wait<0>();
    __syncthreads();
    auto pre = [&](int v) -> cx<T> { return v < n ? ldk(sg.pre + v) : mkc<T>(0, 0); };
    auto in = [&](int v, int t, cx<T> c) -> cx<T> {
      if (v >= n || t >= nt) return mkc<T>(0, 0);
      return cmulc<T>(mkc<T>(stg[(2 * t) * P + v], stg[(2 * t + 1) * P + v]), c);
    };
    auto nopost = [](int) -> cx<T> { return mkc<T>(0, 0); };
    auto none = [](int, int, cx<T>, cx<T>) {};
    const int next = it + gridDim.x;
    // M >= 4L: the n = 2L-1 inputs sit in the first half of the period, the
    // outputs m (and M - m), m < L_j <= M/4, in the first and last quarter
    fft_convolve_n<T, NT, true, 0x00FFu, 0xF00Fu>(A, ST, logM, sg.H, sg.tw, pre, in, nopost, none,
                                                   [&]() { prefetch(next); });
    const T h = sg.scale * T(0.5);
    for (int mm = threadIdx.x; mm < Lj; mm += blockDim.x) {
      const cx<T> ch = ldk(sg.post + mm);
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (t >= nt) break;
        const cx<T> zp = cmulc<T>(A[t * ST + fpad(mm)], ch);
        const cx<T> zm = cmulc<T>(A[t * ST + fpad((M - mm) & (M - 1))], ch);
        // V1 = (Zp + conj(Zm))/2, V2 = (Zp - conj(Zm))/(2i), rows 2(p0 + t), 2(p0 + t) + 1
        cx<T>* __restrict__ V1 = sg.buf_out + (size_t)(2 * (p0 + t)) * Lj;  // V_g[b][m] rows, m fastest
        V1[mm] = mkc<T>((zp.x + zm.x) * h, (zp.y - zm.y) * h);
        if (2 * (p0 + t) + 1 < rows) V1[Lj + mm] = mkc<T>((zp.y + zm.y) * h, (zm.x - zp.x) * h);
      }
    }
    __syncthreads();  // A is rewritten by the next item
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Segmented chirp-z for the alpha sums of scales whose band L_j is small next
// to L (Eqs. (30), (37)).  A chirp-z convolution of length M covers the n =
// 2L-1 outputs at once and costs two FFTs of M >= n + 2 L_j - 2; here the n
// outputs (analysis) or inputs (synthesis) are cut into S segments of P =
// M' - 2 L_j + 2 samples, each a circular convolution of a shorter length M'
// with its own kernel spectrum (the chirp shifted by the segment's first
// sample a_s = s P).  Analysis: one forward FFT of the pre-chirped row, then
// per segment the product with its spectrum and an inverse FFT that yields P
// outputs.  Synthesis (the adjoint): per segment a forward FFT of the
// segment's inputs, products accumulated over the segments in the frequency
// domain, then one inverse FFT.  S + 1 FFTs of M' replace two of M.  A CTA
// runs G = 4096 / M' row pairs side by side, one per group of M'/16 threads.
// ---------------------------------------------------------------------------
// Barrier of thread group g (nthr = M'/16 threads, G = 256 / nthr groups per
// CTA): a warp's own sync for one warp, a named barrier (id 1 + g) for a
// part of the CTA, the CTA barrier for the whole.
__device__ __forceinline__ void seg_group_sync(int nthr, int g) {
  if (nthr >= 256) __syncthreads();
  else if (nthr == 32) __syncwarp();
  else asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(nthr) : "memory");
}

// The analysis kernel branches once per CTA (its segment's length M') to a
// body compiled for that length (FP32 DH plans: M' = 2^9 .. 2^11; others,
// and the FP64 and MW-grid instantiations, take the runtime-length body).
template <typename T, bool ODD, int LOGM>
__device__ __forceinline__ void alpha_ana_seg_body(const CztSeg<T>& sg, const CallPtrs& ptrs, cx<T>* sm) {
  const int logM = LOGM ? LOGM : sg.logM, M = 1 << logM, nthr = M / 16, G = 256 / nthr;
  const int g = threadIdx.x / nthr, tid = threadIdx.x % nthr, ST = fft_smem_elems(M);
  // the groups share no shared memory: each waits for its own threads only
  auto gsync = [&]() { seg_group_sync(nthr, g); };
  cx<T>* Y = sm + g * ST;
  cx<T>* Z = sm + (G + g) * ST;
  const int Lj = sg.Lj, L = sg.L, n = 2 * L - 1, P = sg.P, S = sg.nsegs;
  const int pidx = (blockIdx.x - sg.start) * G + g;  // row pair (complex transform) of this group
  const int rows = sg.N * sg.nb;
  const bool valid = pidx < (ODD ? rows + 1 : rows) / 2, two = !ODD || 2 * pidx + 1 < rows;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);  // nmid == 1 for 9 <= logM <= 12
  const cx<T>* __restrict__ X = sg.buf_in + (size_t)(2 * (valid ? pidx : 0)) * Lj;
  const cx<T>* __restrict__ tw1 = sg.tw + fft_twiddle_level_offset(logM, 1);
  // y_m = (X1 + i X2)_m e^{i pi m^2/n} at position m mod M
  fftg_first_fwd<T>(Y, M, tid, sg.tw, [&](int v) -> cx<T> {
    if (!valid) return mkc<T>(0, 0);
    if (v < Lj) {  // X read once: streaming loads
      const cx<T> x1 = __ldcs(X + v), x2 = __ldcs(X + Lj + v);  // a missing partner: the zero row after the last
      return cmul<T>(mkc<T>(x1.x - x2.y, x1.y + x2.x), ldk(sg.pre + v));
    }
    if (v > M - Lj) {
      const int mm = M - v;
      const cx<T> x1 = __ldcs(X + mm), x2 = __ldcs(X + Lj + mm);
      return cmul<T>(mkc<T>(x1.x + x2.y, x2.x - x1.y), ldk(sg.pre + mm));  // conj(X1) + i conj(X2)
    }
    return mkc<T>(0, 0);
  });
  gsync();
  fftg_stage16<T, false>(Y, M, M / 16, tid, nthr, tw1);
  gsync();
  fftg_inner<T, 0>(Y, Y, M, Rl, tid, nthr, nullptr);
  gsync();
  T* __restrict__ Wb = reinterpret_cast<T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff +
                       (size_t)(2 * (valid ? pidx : 0)) * n;
  for (int s = 0; s < S; ++s) {
    fftg_inner<T, 1>(Y, Z, M, Rl, tid, nthr, sg.H + (size_t)s * M);
    gsync();
    fftg_stage16<T, true>(Z, M, M / 16, tid, nthr, tw1);
    gsync();
    const int as = s * P;
    fftg_last_inv<T>(Z, M, tid, sg.tw, [&](int v, cx<T> y) {
      const int a = as + v;
      if (valid && v < P && a < n) {
        const cx<T> w = cmul<T>(y, ldk(sg.post + a));
        __stcs(Wb + a, w.x);
        if (two) __stcs(Wb + n + a, w.y);
      }
    });
    gsync();  // Z is rewritten by the next segment
  }
}

// CTA `ahead` places later (about one wave): its rows of the layout its
// segment uses (G = 4096 / M' row pairs per CTA, rows 2 p0 .. of `base`
// with `pitch` elements of E per row), asked of L2 ahead of use.
template <typename T, typename E>
__device__ __forceinline__ void seg_prefetch_rows(const CztSeg<T>* __restrict__ segs, int nseg, int ahead,
                                                  const E* base_of_seg_dummy, bool w_rows, const CallPtrs& ptrs) {
  if (threadIdx.x != 0 || blockIdx.x + ahead >= gridDim.x) return;
  const int b2 = blockIdx.x + ahead;
  const CztSeg<T>& s2 = segs[czt_find_seg<T>(segs, nseg, b2)];
  const int G2 = 4096 >> s2.logM, p0 = (b2 - s2.start) * G2, nr = min(2 * G2, s2.N * s2.nb - 2 * p0);
  if (nr <= 0) return;
  (void)base_of_seg_dummy;
  if (!w_rows) {
    prefetch_l2(s2.buf_in + (size_t)(2 * p0) * s2.Lj, (size_t)nr * s2.Lj * sizeof(cx<T>));
  } else {
    const int n = 2 * s2.L - 1;
    const T* W = reinterpret_cast<const T*>(s2.is_phi ? ptrs.Wphi[s2.job] : ptrs.W[s2.job]) + s2.woff;
    prefetch_l2(W + (size_t)(2 * p0) * n, (size_t)nr * n * sizeof(T));
  }
}

template <typename T, bool ODD>
__global__ void __launch_bounds__(256) k_czt_alpha_ana_seg(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs,
                                                           int ahead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  seg_prefetch_rows<T, T>(segs, nseg, ahead, nullptr, false, ptrs);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  if constexpr (sizeof(T) == sizeof(float) && !ODD) {
    switch (sg.logM) {
      case 9: alpha_ana_seg_body<T, ODD, 9>(sg, ptrs, sm); return;
      case 10: alpha_ana_seg_body<T, ODD, 10>(sg, ptrs, sm); return;
      case 11: alpha_ana_seg_body<T, ODD, 11>(sg, ptrs, sm); return;
      default: break;
    }
  }
  alpha_ana_seg_body<T, ODD, 0>(sg, ptrs, sm);
}

template <typename T, bool ODD, int LOGM>
__device__ __forceinline__ void alpha_syn_seg_body(const CztSeg<T>& sg, const CallPtrs& ptrs, cx<T>* sm) {
  const int logM = LOGM ? LOGM : sg.logM, M = 1 << logM, nthr = M / 16, G = 256 / nthr;
  const int g = threadIdx.x / nthr, tid = threadIdx.x % nthr, ST = fft_smem_elems(M);
  auto gsync = [&]() { seg_group_sync(nthr, g); };
  cx<T>* ACC = sm + g * ST;
  cx<T>* B = sm + (G + g) * ST;
  const int Lj = sg.Lj, L = sg.L, n = 2 * L - 1, P = sg.P, S = sg.nsegs;
  const int pidx = (blockIdx.x - sg.start) * G + g;
  const int rows = sg.N * sg.nb;
  const bool valid = pidx < (ODD ? rows + 1 : rows) / 2, two = !ODD || 2 * pidx + 1 < rows;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  const cx<T>* __restrict__ tw1 = sg.tw + fft_twiddle_level_offset(logM, 1);
  const T* __restrict__ Wr = reinterpret_cast<const T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) +
                             sg.woff + (size_t)(2 * (valid ? pidx : 0)) * n;
  // A missing second row (odd row count, MW grid) re-reads the first: the
  // split below recovers the first row's transform whatever its finite
  // partner, and the second is not stored.  (A guarded load here costs a
  // quarter of the kernel's time.)
  const int o2 = two ? n : 0;
  for (int s = 0; s < S; ++s) {
    const int as = s * P;
    // u_p = (W1 + i W2)_{a_s + p} e^{-i pi a^2/n}, p < P
    fftg_first_fwd<T>(B, M, tid, sg.tw, [&](int v) -> cx<T> {
      const int a = as + v;
      if (!valid || v >= P || a >= n) return mkc<T>(0, 0);
      return cmulc<T>(mkc<T>(__ldcs(Wr + a), __ldcs(Wr + o2 + a)), ldk(sg.pre + a));
    });
    gsync();
    fftg_stage16<T, false>(B, M, M / 16, tid, nthr, tw1);
    gsync();
    fftg_inner<T, 2>(B, ACC, M, Rl, tid, nthr, sg.H + (size_t)s * M, s == 0);
    gsync();
  }
  fftg_inner<T, 3>(ACC, ACC, M, Rl, tid, nthr, nullptr);
  gsync();
  fftg_stage16<T, true>(ACC, M, M / 16, tid, nthr, tw1);
  gsync();
  fftg_last_inv<T>(ACC, M, tid, sg.tw, [&](int v, cx<T> y) { ACC[fpad(v)] = y; });
  gsync();
  if (!valid) return;
  const T h = sg.scale * T(0.5);
  cx<T>* __restrict__ V1 = sg.buf_out + (size_t)(2 * pidx) * Lj;  // V_g[b][m] rows, m fastest
  for (int mm = tid; mm < Lj; mm += nthr) {
    const cx<T> ch = ldk(sg.post + mm);
    const cx<T> zp = cmulc<T>(ACC[fpad(mm)], ch);
    const cx<T> zm = cmulc<T>(ACC[fpad((M - mm) & (M - 1))], ch);
    // V1 = (Zp + conj(Zm))/2, V2 = (Zp - conj(Zm))/(2i)
    V1[mm] = mkc<T>((zp.x + zm.x) * h, (zp.y - zm.y) * h);
    if (two) V1[Lj + mm] = mkc<T>((zp.y + zm.y) * h, (zm.x - zp.x) * h);
  }
}

template <typename T, bool ODD>
__global__ void __launch_bounds__(256) k_czt_alpha_syn_seg(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs,
                                                           int ahead) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(smem_raw);
  seg_prefetch_rows<T, T>(segs, nseg, ahead, nullptr, true, ptrs);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  // (the bodies compiled per length measured slower here than this one)
  alpha_syn_seg_body<T, ODD, 0>(sg, ptrs, sm);
}

template <typename T, int NT>  // NT adjacent columns per CTA (the segment's P)
__device__ __forceinline__ void czt_beta_syn_body(const CztSeg<T>& sg, cx<T>* A) {
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, M = 1 << sg.logM, ST = fft_smem_elems(M);
  const int per_g = (Lj + NT - 1) / NT;
  const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, Lj - m0);
  const cx<T>* __restrict__ V = sg.buf_in + (size_t)g * sg.nb * Lj + m0;  // columns m0.. of V_g[b][m]
  auto pref = [&](int v) -> cx<T> { return v < sg.nb ? ldk(sg.pre + v) : mkc<T>(0, 0); };
  auto in = [&](int v, int t, cx<T> c) -> cx<T> {
    if (v >= sg.nb || t >= nt) return mkc<T>(0, 0);
    return cmul<T>(V[(size_t)v * Lj + t], c);
  };
  auto nopost = [](int) -> cx<T> { return mkc<T>(0, 0); };
  auto none = [](int, int, cx<T>, cx<T>) {};
  // inputs b < nb <= 2L <= M/2; outputs m' < L_j and M - m', L_j <= M/4
  fft_convolve_n<T, NT, true, 0x00FFu, 0xF00Fu>(A, ST, sg.logM, sg.H, sg.tw, pref, in, nopost, none, []() {});
  cx<T>* __restrict__ Vh = sg.buf_out + (size_t)g * Lj * Lj + m0;  // columns m0.. of Vhat_g[m'][m]
  const bool pair = NT == 2 && nt == 2 && (Lj & 1) == 0;  // 16-byte aligned column pairs
  for (int mp = threadIdx.x; mp < Lj; mp += blockDim.x) {
    const cx<T> cp = ldk(sg.post + L - 1 + mp), cm = mp > 0 ? ldk(sg.post + L - 1 - mp) : mkc<T>(0, 0);
    cx<T> o[NT];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      const T sigma = ((m0 + t + sg.N - 1) & 1) ? T(-1) : T(1);
      o[t] = cmul<T>(A[t * ST + fpad(mp)], cp);
      if (mp > 0) {
        const cx<T> tm = cmul<T>(A[t * ST + fpad(M - mp)], cm);
        o[t] = mkc<T>(o[t].x + sigma * tm.x, o[t].y + sigma * tm.y);
      }
    }
    cx<T>* __restrict__ vr = Vh + (size_t)mp * Lj;
    if (pair) {
      *reinterpret_cast<float4*>(vr) = make_float4(o[0].x, o[0].y, o[NT - 1].x, o[NT - 1].y);
    } else {
      for (int t = 0; t < nt; ++t) vr[t] = o[t];
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(256, 2) k_czt_beta_syn(const CztSeg<T>* __restrict__ segs, int nseg) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  if (sizeof(T) == sizeof(float) && sg.P == 2) czt_beta_syn_body<T, 2>(sg, A);
  else czt_beta_syn_body<T, 1>(sg, A);
}

// ---------------------------------------------------------------------------
// Beta sums when 4L is the FFT length M (L a power of two): the samples
// beta_b = pi (2b+1)/(4L) lie on the grid 2 pi b / M shifted by pi/(4L), so
//   analysis:  X_b = sum_{|m'|<Lj} (Yhat_{m'} e^{i pi m'/(4L)}) e^{2 pi i m' b/M}
//   synthesis: T_{m'} = e^{-i pi m'/(4L)} sum_{b<2L} (q_b V_b) e^{-2 pi i m' b/M}
// are one FFT each instead of a chirp-z convolution (two FFTs).
// pre: e^{i pi m'/(4L)} at index m' + L - 1; post: q_b (real part), b < 2L.
// ---------------------------------------------------------------------------
// A CTA transforms NT adjacent columns m0.. of one gamma sample (FP32: two),
// so the strided column reads and writes move NT complex values at a time.
// Persistent (items it = blockIdx.x, + gridDim.x, ...): the next item's
// input rows Y_g[m0 + t][.] (contiguous) are staged in shared memory by
// cp.async while the current one is transformed, issued once the current
// item's rows have been scattered into the FFT buffer.  Odd L_j in FP32
// (rows not 16-byte aligned) reads them directly.
template <typename T>
__device__ __forceinline__ bool beta_ana_staged(int Lj) {
  return sizeof(T) == 8 || Lj % 2 == 0;
}

template <typename T, int LOGM>
__global__ void __launch_bounds__(256, 2) k_beta_ana_fft(const CztSeg<T>* __restrict__ segs, int nseg, int total,
                                                         int maxlogM) {
  constexpr int NT = beta_fft_nt(sizeof(T) == 8);
  constexpr int EPC = 16 / (int)sizeof(cx<T>);  // complex values per 16-byte copy
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const int STmax = fft_smem_elems(1 << maxlogM);
  cx<T>* stg = A + NT * STmax;  // [t][m'] rows of the next item, L_j <= M/4
  auto prefetch = [&](int it) {
    if (it < total) {
      const CztSeg<T> sp = segs[czt_find_seg<T>(segs, nseg, it)];
      const int item = it - sp.start, per_g = (sp.Lj + NT - 1) / NT;
      const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, sp.Lj - m0);
      if (beta_ana_staged<T>(sp.Lj)) {
        const cx<T>* Y = sp.buf_in + ((size_t)g * sp.Lj + m0) * sp.Lj;  // nt consecutive rows
        const int nchunk = nt * sp.Lj / EPC;
        for (int i = threadIdx.x; i < nchunk; i += blockDim.x) cp_async16(stg + i * EPC, Y + i * EPC, 16);
      }
    }
    cp_async_commit();
  };
  prefetch(blockIdx.x);
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg, it)];
    const int item = it - sg.start;
    const int Lj = sg.Lj, L = sg.L, logM = LOGM ? LOGM : sg.logM, M = 1 << logM, ST = fft_smem_elems(M);
    const int per_g = (Lj + NT - 1) / NT;
    const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, Lj - m0);
    const bool staged = beta_ana_staged<T>(Lj);
    cp_async_wait<0>();
    __syncthreads();  // staged rows visible; A free
    for (int i = threadIdx.x; i < NT * ST; i += blockDim.x) A[i] = mkc<T>(0, 0);
    __syncthreads();
    const cx<T>* __restrict__ tb = sg.pre + (L - 1);
    for (int t = 0; t < nt; ++t) {
      const int m = m0 + t;
      const T sigma = ((m + sg.N - 1) & 1) ? T(-1) : T(1);
      const cx<T>* __restrict__ Y = sg.buf_in + ((size_t)g * Lj + m) * Lj;  // Y_g[m][.], m' fastest
      for (int mp = threadIdx.x - (Lj - 1); mp < Lj; mp += blockDim.x) {
        const int am = mp < 0 ? -mp : mp;
        cx<T> y = staged ? stg[t * Lj + am] : Y[am];
        if (mp < 0) y = cscale<T>(y, sigma);
        A[t * ST + fpad(fft_pos(mp & (M - 1), logM))] = cmul<T>(y, ldk(tb + mp));
      }
    }
    __syncthreads();
    prefetch(it + gridDim.x);  // stg has been read by every thread
    cx<T>* __restrict__ X = sg.buf_out + (size_t)g * sg.nb * Lj + m0;
    const bool pair = (NT == 2) && (nt == 2) && (Lj % 2 == 0);  // 16-byte aligned column pairs
    fft_inverse_to_n<T, NT, 0x00FFu>(A, ST, logM, sg.tw, [&](int v, const cx<T>* y) {  // v < 2L = M/2
      if (v < sg.nb) {
        if (pair) {
          *reinterpret_cast<float4*>(X + (size_t)v * Lj) = *reinterpret_cast<const float4*>(y);
        } else {
          for (int t = 0; t < nt; ++t) X[(size_t)v * Lj + t] = y[t];
        }
      }
    });
  }
  cp_async_wait<0>();
}

// shared memory of k_beta_ana_fft: NT transforms of the largest length and
// the staged input rows (NT rows of at most L = M/4 values)
template <typename T>
size_t beta_ana_fft_smem(int maxlogM) {
  constexpr int NT = beta_fft_nt(sizeof(T) == 8);
  return (size_t)NT * (fft_smem_elems(1 << maxlogM) + ((size_t)1 << (maxlogM - 2))) * sizeof(cx<T>);
}

// Persistent (items it = blockIdx.x, + gridDim.x, ...): the strided column
// rows of the next item (16 bytes per row b: the NT complex values of
// columns m0..) are staged in shared memory by cp.async while the current
// one is transformed, issued as soon as the current item's first FFT stage
// has read its inputs.  Items whose rows are not 16-byte aligned (odd L_j,
// a last single column) read them directly.
template <typename T>
__device__ __forceinline__ bool beta_syn_staged(int Lj, int nt) {
  constexpr int NT = beta_fft_nt(sizeof(T) == 8);
  return NT * sizeof(cx<T>) == 16 && nt == NT && (sizeof(T) == 8 || Lj % 2 == 0);
}

template <typename T, int LOGM>
__global__ void __launch_bounds__(256, 2) k_beta_syn_fft(const CztSeg<T>* __restrict__ segs, int nseg, int total,
                                                         int maxlogM) {
  constexpr int NT = beta_fft_nt(sizeof(T) == 8);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  const int STmax = fft_smem_elems(1 << maxlogM);
  cx<T>* stg = A + NT * STmax;  // [b][NT] rows of the next item
  auto prefetch = [&](int it) {
    if (it < total) {
      const CztSeg<T> sp = segs[czt_find_seg<T>(segs, nseg, it)];
      const int item = it - sp.start, per_g = (sp.Lj + NT - 1) / NT;
      const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, sp.Lj - m0);
      if (beta_syn_staged<T>(sp.Lj, nt)) {
        const cx<T>* V = sp.buf_in + (size_t)g * sp.nb * sp.Lj + m0;
        for (int v = threadIdx.x; v < sp.nb; v += blockDim.x) cp_async16(stg + v * NT, V + (size_t)v * sp.Lj, 16);
      }
    }
    cp_async_commit();
  };
  prefetch(blockIdx.x);
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg, it)];
    const int item = it - sg.start;
    const int Lj = sg.Lj, L = sg.L, logM = LOGM ? LOGM : sg.logM, M = 1 << logM, ST = fft_smem_elems(M);
    const int per_g = (Lj + NT - 1) / NT;
    const int g = item / per_g, m0 = (item % per_g) * NT, nt = min(NT, Lj - m0);
    const bool staged = beta_syn_staged<T>(Lj, nt);
    const bool pair = (NT == 2) && (nt == 2) && (Lj % 2 == 0);
    const cx<T>* __restrict__ V = sg.buf_in + (size_t)g * sg.nb * Lj + m0;  // columns m0.. of V_g[b][m]
    const cx<T>* __restrict__ q = sg.post;
    cp_async_wait<0>();
    __syncthreads();  // staged rows visible; A free
    fft_forward_from_n<T, NT, 0x00FFu>(  // inputs b < 2L = M/2
        A, ST, logM, sg.tw,
        [&](int v, cx<T>* x) {
          if (v >= sg.nb) {
#pragma unroll
            for (int t = 0; t < NT; ++t) x[t] = mkc<T>(0, 0);
            return;
          }
          const T qv = ldk(q + v).x;
          if (staged) {
#pragma unroll
            for (int t = 0; t < NT; ++t) x[t] = cscale<T>(stg[v * NT + t], qv);
          } else if (pair) {
            const float4 u = *reinterpret_cast<const float4*>(V + (size_t)v * Lj);
            const cx<T>* uu = reinterpret_cast<const cx<T>*>(&u);
#pragma unroll
            for (int t = 0; t < NT; ++t) x[t] = cscale<T>(uu[t], qv);
          } else {
#pragma unroll
            for (int t = 0; t < NT; ++t) x[t] = t < nt ? cscale<T>(V[(size_t)v * Lj + t], qv) : mkc<T>(0, 0);
          }
        },
        [&]() { prefetch(it + gridDim.x); });  // stg has been read by every thread
    const cx<T>* __restrict__ tb = sg.pre + (L - 1);
    cx<T>* __restrict__ Vh = sg.buf_out + (size_t)g * Lj * Lj + m0;  // columns m0.. of Vhat_g[m'][m]
    for (int mp = threadIdx.x; mp < Lj; mp += blockDim.x) {
      cx<T> o[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        const T sigma = ((m0 + t + sg.N - 1) & 1) ? T(-1) : T(1);
        o[t] = cmulc<T>(A[t * ST + fpad(fft_pos(mp, logM))], ldk(tb + mp));
        if (mp > 0) {
          const cx<T> tm = cmulc<T>(A[t * ST + fpad(fft_pos(M - mp, logM))], ldk(tb - mp));
          o[t] = mkc<T>(o[t].x + sigma * tm.x, o[t].y + sigma * tm.y);
        }
      }
      if (pair) {
        *reinterpret_cast<float4*>(Vh + (size_t)mp * Lj) = *reinterpret_cast<const float4*>(o);
      } else {
        for (int t = 0; t < nt; ++t) Vh[(size_t)mp * Lj + t] = o[t];
      }
    }
  }
  cp_async_wait<0>();
}

// shared memory of k_beta_syn_fft: NT transforms of the largest length and
// the staged rows (2L = M/2 rows of 16 bytes)
template <typename T>
size_t beta_syn_fft_smem(int maxlogM) {
  return (size_t)beta_fft_nt(sizeof(T) == 8) * fft_smem_elems(1 << maxlogM) * sizeof(cx<T>) +
         ((size_t)1 << (maxlogM - 1)) * 16;
}

// ---------------------------------------------------------------------------
// Beta sums as half-length transforms (L a power of two, L >= 16).  With the
// fold Yhat_{-m'} = sigma Yhat_{m'} every beta sum is a cosine or sine
// series in m' evaluated at beta_b = pi (2b+1) / (2N), N = 2L, i.e. a complex
// DCT-III / DST-III (analysis) or DCT-II / DST-II (synthesis quadrature) of
// length N, each computed with one complex FFT of length N (the length-4L
// FFT of k_beta_*_fft computes the same samples with half its output unused):
//   analysis:  Z_k = (Yhat_k - sigma i Yhat_{N-k}) e^{i pi k/(2N)},
//              u_n = sum_k Z_k e^{2 pi i k n/N},
//              X_b(n) = s_b u_n with b(n) = 2n (n < N/2), 2N-1-2n (n >= N/2),
//              s_b = (-1)^b if sigma = -1, else 1;
//   synthesis: y_v = sgn_v q_b(v) V_b(v) (sgn_v = -1 for sigma = -1, v >= N/2),
//              Y = sum_v y_v e^{-2 pi i k v/N},
//              Vhat_k = e^{-i pi k/(2N)} Y_k + sigma e^{i pi k/(2N)} Y_{N-k} (k >= 1),
//              Vhat_0 = Y_0 (sigma = +1; for sigma = -1 the m' = 0 entry meets
//              Delta^l_{0m} Delta^l_{0n} = 0 in the contraction and is set to 0).
// A CTA runs G = 4096/N transforms side by side, one per group of N/16
// threads (adjacent columns m of one gamma sample), with the thread-group
// stages of fft16.cuh.  All shared-memory reads after the FFT are in natural
// position order (position p holds frequency fft_rev(p); its negation
// partner N - fft_rev(p) sits in a descending run of positions), and each
// output row gets the G columns in one contiguous store.  Persistent: the next
// item's input is staged by cp.async while the current one is transformed.
// pre: e^{i pi m'/(4L)} at index m' + L - 1 (|m'| < L); post: q_b (real part), b < 2L.
// ---------------------------------------------------------------------------

// Frequency held at position p after the forward stages (inverse of fft_pos).
__device__ __forceinline__ int fft_rev(int p, int logM) {
  const int a = logM >> 2, b = logM & 3;
  int f = 0;
  for (int i = 0; i < a; ++i) f |= ((p >> (logM - 4 * (i + 1))) & 15) << (4 * i);
  if (b) f |= (p & ((1 << b) - 1)) << (4 * a);
  return f;
}

// e^{i pi k/(2N)}, k in [0, N), from the table of e^{i pi m'/(4L)}, |m'| < L = N/2
// (k > L: i e^{i pi (k - 2L)/(4L)}; k = L never multiplies a nonzero value).
template <typename T>
__device__ __forceinline__ cx<T> dct_twiddle(const cx<T>* __restrict__ tb, int k, int L) {
  if (k < L) return ldk(tb + k);
  if (k == L) return mkc<T>(0, 0);
  const cx<T> t = ldk(tb + (k - 2 * L));
  return mkc<T>(-t.y, t.x);
}

constexpr int kDctSpan = 4096;  // G * N: transforms per CTA times their length

template <typename T>
size_t beta_dct_smem(bool syn) {
  // FFT buffers (G transforms) + staged input: analysis G rows of at most N/2,
  // synthesis G columns of N samples
  return ((size_t)fft_smem_elems(kDctSpan) + (syn ? kDctSpan : kDctSpan / 2)) * sizeof(cx<T>);
}

template <typename T>
__device__ __forceinline__ bool beta_dct_ana_staged(int Lj) {
  return sizeof(T) == 8 || Lj % 2 == 0;  // 16-byte chunks of the contiguous rows
}

// LOGN > 0: every segment of the launch has transforms of length 2^LOGN (a
// compile-time length lets the stage loops and index maps fold); 0: any.
template <typename T, int LOGN>
__global__ void __launch_bounds__(256) k_beta_ana_dct(const CztSeg<T>* __restrict__ segs, int nseg, int total) {
  constexpr int EPC = 16 / (int)sizeof(cx<T>);
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stg = A + fft_smem_elems(kDctSpan);  // [gi][Lj] rows of the next item
  const int tid = threadIdx.x;
  auto geom = [&](const CztSeg<T>& sp, int it, int& logN, int& G, int& g, int& m0, int& nt) {
    logN = LOGN ? LOGN : sp.logM - 1;
    G = kDctSpan >> logN;
    const int item = it - sp.start, per_g = (sp.Lj + G - 1) / G;
    g = item / per_g;
    m0 = (item % per_g) * G;
    nt = min(G, sp.Lj - m0);
  };
  auto prefetch = [&](int it) {
    if (it < total) {
      const CztSeg<T> sp = segs[czt_find_seg<T>(segs, nseg, it)];
      int logN, G, g, m0, nt;
      geom(sp, it, logN, G, g, m0, nt);
      if (beta_dct_ana_staged<T>(sp.Lj)) {
        const cx<T>* Y = sp.buf_in + ((size_t)g * sp.Lj + m0) * sp.Lj;  // nt consecutive rows
        const int nchunk = nt * sp.Lj / EPC;
        for (int i = tid; i < nchunk; i += blockDim.x) cp_async16(stg + i * EPC, Y + i * EPC, 16);
      }
    }
    cp_async_commit();
  };
  prefetch(blockIdx.x);
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg, it)];
    int logN, G, g, m0, nt;
    geom(sg, it, logN, G, g, m0, nt);
    const int Nn = 1 << logN, nthr = Nn >> 4, gi = tid / nthr, tg = tid % nthr, ST = fft_smem_elems(Nn);
    const int Lj = sg.Lj, L = sg.L;
    const bool staged = beta_dct_ana_staged<T>(Lj);
    const cx<T>* __restrict__ tb = sg.pre + (L - 1);
    const int m = m0 + gi;
    const T sigma = ((m + sg.N - 1) & 1) ? T(-1) : T(1);
    const cx<T>* __restrict__ Yg = sg.buf_in + ((size_t)g * Lj + m) * Lj;
    cx<T>* Ag = A + gi * ST;
    cp_async_wait<0>();
    __syncthreads();  // staged rows visible; A free
    int Rl, nmid;
    fft_schedule(logN, Rl, nmid);
    auto yhat = [&](int u) -> cx<T> {
      if (u >= Lj || gi >= nt) return mkc<T>(0, 0);
      return staged ? stg[gi * Lj + u] : Yg[u];
    };
    // conj(Z_v): the forward stages then give the conjugate of the inverse transform
    fftg_first_fwd<T>(Ag, Nn, tg, sg.tw, [&](int v) -> cx<T> {
      const cx<T> a = yhat(v), b = yhat(Nn - v);
      const cx<T> z = mkc<T>(a.x + sigma * b.y, a.y - sigma * b.x);  // a - sigma i b
      return cconj<T>(cmul<T>(z, dct_twiddle<T>(tb, v, L)));
    });
    __syncthreads();
    prefetch(it + gridDim.x);  // every staged value has been read
    int S = Nn >> 4;
    for (int s = 0; s < nmid; ++s) {
      fftg_stage16<T, false>(Ag, Nn, S, tg, nthr, sg.tw + fft_twiddle_level_offset(logN, s + 1));
      __syncthreads();
      S >>= 4;
    }
    fftg_inner<T, 0>(Ag, Ag, Nn, Rl, tg, nthr, nullptr);
    __syncthreads();
    // X_b(n) = s_b conj(A[pos]) for the position p holding n; G columns per row
    cx<T>* __restrict__ X = sg.buf_out + (size_t)g * sg.nb * Lj + m0;
    // FP32, a compile-time length, all G columns present and 16-byte aligned
    // rows: the G columns of a row leave as G/2 16-byte stores (8-byte
    // stores scattered over rows fill a quarter of each sector)
    constexpr int GC = LOGN > 0 ? (kDctSpan >> LOGN) : 0;
    constexpr bool PAIRS = sizeof(T) == sizeof(float) && GC >= 2;
    const bool pair_st = PAIRS && nt == GC && (Lj & 1) == 0;
    for (int p = tid; p < Nn; p += blockDim.x) {
      const int n = fft_rev(p, logN);
      const int b = n < (Nn >> 1) ? 2 * n : 2 * Nn - 1 - 2 * n;
      if (b >= sg.nb) continue;
      cx<T>* xr = X + (size_t)b * Lj;
      if (pair_st) {
        const T s0 = (((m0 + sg.N - 1) & 1) && (b & 1)) ? T(-1) : T(1);
        const T s1 = (b & 1) ? -s0 : s0;  // odd columns m0 + 2k + 1 have the other parity
#pragma unroll
        for (int k = 0; k < GC / 2; ++k) {
          const cx<T> u0 = A[(2 * k) * ST + fpad(p)], u1 = A[(2 * k + 1) * ST + fpad(p)];
          reinterpret_cast<float4*>(xr)[k] = make_float4(s0 * u0.x, -s0 * u0.y, s1 * u1.x, -s1 * u1.y);
        }
        continue;
      }
      for (int t = 0; t < nt; ++t) {
        const T sg_t = (((m0 + t + sg.N - 1) & 1) && (b & 1)) ? T(-1) : T(1);
        const cx<T> u = A[t * ST + fpad(p)];
        xr[t] = mkc<T>(sg_t * u.x, -sg_t * u.y);
      }
    }
  }
  cp_async_wait<0>();
}

template <typename T, int LOGN>
__global__ void __launch_bounds__(256) k_beta_syn_dct(const CztSeg<T>* __restrict__ segs, int nseg, int total) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* A = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* stg = A + fft_smem_elems(kDctSpan);  // [gi][v]: column gi in FFT input order
  const int tid = threadIdx.x;
  auto geom = [&](const CztSeg<T>& sp, int it, int& logN, int& G, int& g, int& m0, int& nt) {
    logN = LOGN ? LOGN : sp.logM - 1;
    G = kDctSpan >> logN;
    const int item = it - sp.start, per_g = (sp.Lj + G - 1) / G;
    g = item / per_g;
    m0 = (item % per_g) * G;
    nt = min(G, sp.Lj - m0);
  };
  // column t of V_g[b][m0 + t], b < N, staged at v(b) = b/2 (b even), N - 1 - (b-1)/2 (b odd):
  // at stg[t N + v], or, for an even number G of FP32 columns per CTA (a
  // compile-time length), in column pairs at stg[(t/2) 2N + 2 v + t%2] so
  // that one 16-byte copy moves a pair of columns of a row
  constexpr int GC = LOGN > 0 ? (kDctSpan >> LOGN) : 0;
  constexpr bool PAIRS = sizeof(T) == sizeof(float) && GC >= 2;
  auto sidx = [&](int t, int v, int Nn) { return PAIRS ? (t >> 1) * 2 * Nn + 2 * v + (t & 1) : t * Nn + v; };
  auto prefetch = [&](int it) {
    if (it < total) {
      const CztSeg<T> sp = segs[czt_find_seg<T>(segs, nseg, it)];
      int logN, G, g, m0, nt;
      geom(sp, it, logN, G, g, m0, nt);
      const int Nn = 1 << logN;
      const cx<T>* V = sp.buf_in + (size_t)g * sp.nb * sp.Lj + m0;
      if (PAIRS && nt == GC && (sp.Lj & 1) == 0) {  // 16-byte aligned column pairs
        for (int i = tid; i < Nn * (GC / 2); i += blockDim.x) {
          const int k = i / Nn, b = i - k * Nn;
          const int v = (b & 1) ? Nn - 1 - (b >> 1) : (b >> 1);
          cp_async16(stg + k * 2 * Nn + 2 * v, V + (size_t)b * sp.Lj + 2 * k, 16);
        }
      } else {
        for (int i = tid; i < nt * Nn; i += blockDim.x) {
          const int t = i / Nn, b = i - t * Nn;
          const int v = (b & 1) ? Nn - 1 - (b >> 1) : (b >> 1);
          cp_async_ca<sizeof(cx<T>)>(stg + sidx(t, v, Nn), V + (size_t)b * sp.Lj + t);
        }
      }
    }
    cp_async_commit();
  };
  prefetch(blockIdx.x);
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg, it)];
    int logN, G, g, m0, nt;
    geom(sg, it, logN, G, g, m0, nt);
    const int Nn = 1 << logN, nthr = Nn >> 4, gi = tid / nthr, tg = tid % nthr, ST = fft_smem_elems(Nn);
    const int Lj = sg.Lj, L = sg.L;
    const T sigma = ((m0 + gi + sg.N - 1) & 1) ? T(-1) : T(1);
    const cx<T>* __restrict__ q = sg.post;
    cx<T>* Ag = A + gi * ST;
    cp_async_wait<0>();
    __syncthreads();
    int Rl, nmid;
    fft_schedule(logN, Rl, nmid);
    fftg_first_fwd<T>(Ag, Nn, tg, sg.tw, [&](int v) -> cx<T> {
      if (gi >= nt) return mkc<T>(0, 0);
      const int b = v < (Nn >> 1) ? 2 * v : 2 * (Nn - 1 - v) + 1;
      const T w = ldk(q + b).x * ((sigma < T(0) && v >= (Nn >> 1)) ? T(-1) : T(1));
      return cscale<T>(stg[sidx(gi, v, Nn)], w);
    });
    __syncthreads();
    prefetch(it + gridDim.x);
    int S = Nn >> 4;
    for (int s = 0; s < nmid; ++s) {
      fftg_stage16<T, false>(Ag, Nn, S, tg, nthr, sg.tw + fft_twiddle_level_offset(logN, s + 1));
      __syncthreads();
      S >>= 4;
    }
    fftg_inner<T, 0>(Ag, Ag, Nn, Rl, tg, nthr, nullptr);
    __syncthreads();
    const cx<T>* __restrict__ tb = sg.pre + (L - 1);
    cx<T>* __restrict__ Vh = sg.buf_out + (size_t)g * Lj * Lj + m0;  // row k of Vhat_g[m'][m]
    const bool pair_st = sizeof(T) == sizeof(float) && GC >= 2 && nt == GC && (Lj & 1) == 0;
    for (int p = tid; p < Nn; p += blockDim.x) {
      const int k = fft_rev(p, logN);
      if (k >= Lj) continue;
      const int pp = fft_pos((Nn - k) & (Nn - 1), logN);
      const cx<T> w = cconj<T>(ldk(tb + k));  // e^{-i pi k/(2N)}
      cx<T>* vr = Vh + (size_t)k * Lj;
      auto value = [&](int t) -> cx<T> {
        const T sg_t = ((m0 + t + sg.N - 1) & 1) ? T(-1) : T(1);
        const cx<T> yk = A[t * ST + fpad(p)], ynk = A[t * ST + fpad(pp)];
        if (k == 0) return sg_t > T(0) ? yk : mkc<T>(0, 0);
        const cx<T> a = cmul<T>(w, yk), c = cmul<T>(cconj<T>(w), ynk);
        return mkc<T>(a.x + sg_t * c.x, a.y + sg_t * c.y);
      };
      if (pair_st) {  // the G columns of a row as G/2 16-byte stores
#pragma unroll
        for (int q2 = 0; q2 < GC / 2; ++q2) {
          const cx<T> o0 = value(2 * q2), o1 = value(2 * q2 + 1);
          reinterpret_cast<float4*>(vr)[q2] = make_float4(o0.x, o0.y, o1.x, o1.y);
        }
      } else {
        for (int t = 0; t < nt; ++t) vr[t] = value(t);
      }
    }
  }
  cp_async_wait<0>();
}

// ---------------------------------------------------------------------------
// Direct evaluation of the alpha sums for scales with a small band-limit
// L_j <= kDirectMax: the chirp-z cost does not shrink with L_j (the output
// grid has 2L-1 points for every scale) while a direct sum costs ~L_j per
// output.  Twiddles e^{i m alpha_a} advance by one complex product per step
// of m (or a) and are re-read exactly from the root table every 16 steps.
// ---------------------------------------------------------------------------
constexpr int kDirectMax = kDirectMaxLj;

// W[row][a] = X_0 + 2 sum_{m=1}^{Lj-1} Re(X_m e^{2 pi i m a / n})   (Eq. (30), Hermitian in m)
// as a small matrix product W = A B over k < K = 2 Lj - 1 with
//   A[row] = (X_0.x, X_1.x, X_1.y, X_2.x, ...),
//   B[.][a] = (1, 2 cos(2 pi a/n), -2 sin(2 pi a/n), 2 cos(4 pi a/n), ...).
// A CTA owns kAgCols consecutive samples a and kAgChunk rows: it builds its
// B tile once in shared memory from the exact root table (index m a mod n
// advanced by additions), then per pass of kAgRows rows stages A and
// accumulates a register tile of 8 rows x 4 samples per thread, samples
// lane + 32 i so that every store of a warp is one 128-byte line.  Layouts:
// B[k][lane][i] (one 16-byte load per k), A[k][row].  FP64 plans only (FP32
// plans run the tensor-core kernels of alpha_tc.cu).
template <typename T>
__global__ void __launch_bounds__(256) k_alpha_ana_direct(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs) {
  static_assert(sizeof(T) == sizeof(double), "FP32 plans use the tensor-core kernels");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int KMAX = 2 * kDirectMaxLjAna - 1;
  constexpr int AW = 1;                     // stored copies of each A value
  T* Bs = reinterpret_cast<T*>(smem_raw);  // [KMAX][32][4]
  T* As = Bs + KMAX * kAgCols;              // [KMAX][kAgRows][AW]
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, n = 2 * L - 1, K = 2 * Lj - 1;
  const int ntile = (n + kAgCols - 1) / kAgCols;
  const int a0 = (item % ntile) * kAgCols;
  const int nrows = sg.N * sg.nb, rbeg = (item / ntile) * kAgChunk, rend = min(nrows, rbeg + kAgChunk);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const cx<T>* __restrict__ root = sg.pre;  // e^{2 pi i u / n}, u < n
  T* __restrict__ Wb = reinterpret_cast<T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff;
  if (K <= 0) {  // empty scale: W = 0
    for (int r = rbeg; r < rend; ++r)
      for (int c = t; c < kAgCols; c += blockDim.x)
        if (a0 + c < n) Wb[(size_t)r * n + a0 + c] = T(0);
    return;
  }
  // B tile: thread t fills sample c = t % kAgCols for m = 1 + t / kAgCols, step 256 / kAgCols
  {
    constexpr int MS = 256 / kAgCols;
    const int c = t % kAgCols, a = a0 + c;
    const int pos = (c & 31) * 4 + (c >> 5);  // [lane][i] of sample c = lane + 32 i
    const bool ok = a < n;
    if (t < kAgCols) Bs[pos] = ok ? T(1) : T(0);
    int m = 1 + t / kAgCols;
    int u = ok ? (int)(((long long)m * a) % n) : 0;
    const int du = ok ? (int)(((long long)MS * a) % n) : 0;
#pragma unroll 8
    for (; m < Lj; m += MS) {  // unrolled: the root loads of 8 steps are in flight together
      const cx<T> e = ok ? ldk(root + u) : mkc<T>(0, 0);
      Bs[(2 * m - 1) * kAgCols + pos] = T(2) * e.x;
      Bs[(2 * m) * kAgCols + pos] = T(-2) * e.y;
      u += du;
      if (u >= n) u -= n;
    }
  }
  for (int r0 = rbeg; r0 < rend; r0 += kAgRows) {
    const int nr = min(kAgRows, rend - r0);
    __syncthreads();  // B tile written / previous pass done with As
#pragma unroll 4
    for (int i = t; i < kAgRows * Lj; i += blockDim.x) {
      const int m = i / kAgRows, r = i % kAgRows;  // consecutive threads: consecutive rows (no bank conflicts)
      const cx<T> x = r < nr ? sg.buf_in[(size_t)(r0 + r) * Lj + m] : mkc<T>(0, 0);
      const int k1 = m == 0 ? 0 : 2 * m - 1;
#pragma unroll
      for (int d = 0; d < AW; ++d) As[(k1 * kAgRows + r) * AW + d] = x.x;
      if (m > 0) {
#pragma unroll
        for (int d = 0; d < AW; ++d) As[((k1 + 1) * kAgRows + r) * AW + d] = x.y;
      }
    }
    __syncthreads();
    T out[8][4];
    {
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int i = 0; i < 4; ++i) out[r][i] = T(0);
      const T* __restrict__ ap = As + 8 * w;
      const T* __restrict__ bp = Bs + 4 * lane;
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        T av[8], bv[4];
#pragma unroll
        for (int r = 0; r < 8; ++r) av[r] = ap[r];
#pragma unroll
        for (int i = 0; i < 4; ++i) bv[i] = bp[i];
#pragma unroll
        for (int r = 0; r < 8; ++r)
#pragma unroll
          for (int i = 0; i < 4; ++i) out[r][i] = fma(av[r], bv[i], out[r][i]);
        ap += kAgRows;
        bp += kAgCols;
      }
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int row = 8 * w + r;
      if (row < nr) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int a = a0 + lane + 32 * i;
          if (a < n) Wb[(size_t)(r0 + row) * n + a] = out[r][i];
        }
      }
    }
  }
}

// V[row][m] = (2 pi / n) sum_{a<n} W[row][a] e^{-2 pi i m a / n}, m < Lj   (Eq. (37))
// A CTA takes R = 32 / sizeof(T) rows, staged in shared memory as one 32-byte
// line per sample a (Ws[a][r]) so that a lane reads all R rows with two
// 16-byte loads; loads are issued in unrolled batches (rows have odd length,
// so neither 16-byte copies nor TMA tiles apply).  Warp w sums the a-range
// chunk w; its lanes are (sub, m) with P = 32 / Lj lanes per m splitting the
// chunk further.  Partials are reduced over sub by shuffles when Lj divides
// 32, then over the chunks in shared memory.
// FP64 plans only (FP32 plans run the tensor-core kernels of alpha_tc.cu).
template <typename T>
__device__ __forceinline__ void syn_direct_line(const T* p, T (&x)[32 / sizeof(T)]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  x[0] = a.x; x[1] = a.y; x[2] = b.x; x[3] = b.y;
}

template <typename T>
__global__ void __launch_bounds__(256) k_alpha_syn_direct(const CztSeg<T>* __restrict__ segs, int nseg, CallPtrs ptrs) {
  static_assert(sizeof(T) == sizeof(double), "FP32 plans use the tensor-core kernels");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  constexpr int R = 32 / sizeof(T);
  constexpr int U = 4;  // samples per thread per load batch (R * U loads in flight)
  const CztSeg<T> sg = segs[czt_find_seg<T>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, L = sg.L, n = 2 * L - 1;
  const int nrows = sg.N * sg.nb, row0 = item * R, nr = min(R, nrows - row0);
  T* Ws = reinterpret_cast<T*>(smem_raw);  // [n][R], later the partials
  const T* __restrict__ Wb = reinterpret_cast<const T*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff +
                             (size_t)row0 * n;
  const int tid = threadIdx.x;
  for (int a0 = 0; a0 < n; a0 += U * 256) {
    T x[U][R];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + u * 256 + tid;
#pragma unroll
      for (int r = 0; r < R; ++r) x[u][r] = (a < n && r < nr) ? __ldg(Wb + (size_t)r * n + a) : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int a = a0 + u * 256 + tid;
      if (a < n) {
        double2* d = reinterpret_cast<double2*>(Ws + (size_t)a * R);
        d[0] = make_double2(x[u][0], x[u][1]);
        d[1] = make_double2(x[u][2], x[u][3]);
      }
    }
  }
  __syncthreads();
  const cx<T>* __restrict__ root = sg.pre;  // e^{2 pi i t / n}
  const int warp = tid >> 5, lane = tid & 31;
  const int P = 32 / Lj, m = lane % Lj, sub = lane / Lj;
  const bool active = sub < P;
  cx<T> acc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) acc[r] = mkc<T>(0, 0);
  if (active) {
    const int c_lo = (int)(((long long)n * warp) / 8), c_hi = (int)(((long long)n * (warp + 1)) / 8);
    const int a_lo = c_lo + (int)(((long long)(c_hi - c_lo) * sub) / P);
    const int a_hi = c_lo + (int)(((long long)(c_hi - c_lo) * (sub + 1)) / P);
    const cx<T> st = cconj<T>(ldk(root + m));
    cx<T> w = mkc<T>(1, 0);
    for (int a = a_lo; a < a_hi; ++a) {
      if (((a - a_lo) & 15) == 0) w = cconj<T>(ldk(root + (m * a) % n));
      T x[R];
      syn_direct_line<T>(Ws + (size_t)a * R, x);
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acc[r].x = fma(x[r], w.x, acc[r].x);
        acc[r].y = fma(x[r], w.y, acc[r].y);
      }
      w = cmul<T>(w, st);
    }
  }
  // in-warp reduction over sub (lanes m, m + Lj, m + 2 Lj, ...) when Lj | 32
  const bool shfl = (32 % Lj) == 0;
  if (shfl) {
    for (int off = Lj; off < 32; off <<= 1) {
#pragma unroll
      for (int r = 0; r < R; ++r) {
        acc[r].x += __shfl_xor_sync(0xffffffffu, acc[r].x, off);
        acc[r].y += __shfl_xor_sync(0xffffffffu, acc[r].y, off);
      }
    }
  }
  const int nchunk = shfl ? 8 : 8 * P;
  __syncthreads();  // Ws is reused for the partials [nchunk][Lj][R]
  cx<T>* part = reinterpret_cast<cx<T>*>(smem_raw);
  if (active && (!shfl || sub == 0)) {
    const int c = shfl ? warp : warp * P + sub;
#pragma unroll
    for (int r = 0; r < R; ++r) part[((size_t)c * Lj + m) * R + r] = acc[r];
  }
  __syncthreads();
  for (int i = tid; i < Lj * R; i += blockDim.x) {
    const int mm = i / R, r = i % R;
    if (r >= nr) continue;
    cx<T> s = mkc<T>(0, 0);
    for (int c2 = 0; c2 < nchunk; ++c2) s = cadd<T>(s, part[((size_t)c2 * Lj + mm) * R + r]);
    sg.buf_out[(size_t)(row0 + r) * Lj + mm] = cscale<T>(s, sg.scale);
  }
}

// shared memory of k_alpha_syn_direct for band-limits up to L: the staged
// rows, or the partials (at most 256 x R complex) if larger
template <typename T>
size_t alpha_syn_direct_smem(int L) {
  const size_t n = 2 * (size_t)L - 1;
  const size_t rows = n * 32, parts = (size_t)256 * (32 / sizeof(T)) * sizeof(cx<T>);
  return rows > parts ? rows : parts;
}

// CTAs of a kernel resident at once on this device (the grid of a
// persistent kernel; the look-ahead of the L2 prefetches).
template <typename T, typename K>
int alpha_czt_grid(K kernel, size_t smem) {
  // cached per (device, kernel, shared-memory size)
  struct Entry {
    int dev;
    const void* fn;
    size_t smem;
    int grid;
  };
  static std::mutex mu;
  static std::vector<Entry> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const void* fn = reinterpret_cast<const void*>(kernel);
  {
    std::lock_guard<std::mutex> lk(mu);
    for (const Entry& e : cache)
      if (e.dev == dev && e.fn == fn && e.smem == smem) return e.grid;
  }
  int sms = 0, per = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, 256, smem);
  const int g = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
  std::lock_guard<std::mutex> lk(mu);
  cache.push_back({dev, fn, smem, g});
  return g;
}

template <typename T>
void launch_czt_impl(int kind, const CztSeg<T>* segs, int nseg, int total_items, int maxlogM,
                     const CallPtrs& ptrs, cudaStream_t st, int uniform_logM = 0) {
  if (total_items <= 0) return;
  const bool odd = (kind & CZT_ODD_ROWS) != 0;
  kind &= ~CZT_ODD_ROWS;
  // FP32 launches whose segments share one transform length of 2^11 .. 2^13
  // take the kernels compiled for that length
  const int ulog = (sizeof(T) == sizeof(float) && uniform_logM >= 11 && uniform_logM <= 13) ? uniform_logM : 0;
  if (kind == CZT_ALPHA_ANA) {
    auto k = odd ? k_czt_alpha_ana<T, true, 0> : k_czt_alpha_ana<T, false, 0>;
    if constexpr (sizeof(T) == sizeof(float)) {
      if (!odd && ulog == 11) k = k_czt_alpha_ana<T, false, 11>;
      if (!odd && ulog == 12) k = k_czt_alpha_ana<T, false, 12>;
      if (!odd && ulog == 13) k = k_czt_alpha_ana<T, false, 13>;
    }
    const size_t sm = alpha_czt_smem<T>(maxlogM, false);
    k<<<total_items, 256, sm, st>>>(segs, nseg, maxlogM, ptrs, alpha_czt_grid<T>(k, sm));
    return;
  }
  if (kind == CZT_ALPHA_ANA_SEG) {
    auto k = odd ? k_czt_alpha_ana_seg<T, true> : k_czt_alpha_ana_seg<T, false>;
    k<<<total_items, 256, alpha_seg_smem<T>(), st>>>(segs, nseg, ptrs, alpha_czt_grid<T>(k, alpha_seg_smem<T>()));
    return;
  }
  if (kind == CZT_ALPHA_SYN_SEG) {
    auto k = odd ? k_czt_alpha_syn_seg<T, true> : k_czt_alpha_syn_seg<T, false>;
    k<<<total_items, 256, alpha_seg_smem<T>(), st>>>(segs, nseg, ptrs, alpha_czt_grid<T>(k, alpha_seg_smem<T>()));
    return;
  }
  if (kind == CZT_ALPHA_SYN) {
    const size_t sm = alpha_czt_smem<T>(maxlogM, true);
    auto k = k_czt_alpha_syn<T, 0>;
    if constexpr (sizeof(T) == sizeof(float)) {
      if (ulog == 11) k = k_czt_alpha_syn<T, 11>;
      if (ulog == 12) k = k_czt_alpha_syn<T, 12>;
      if (ulog == 13) k = k_czt_alpha_syn<T, 13>;
    }
    const int g = std::min(total_items, alpha_czt_grid<T>(k, sm));
    k<<<g, 256, sm, st>>>(segs, nseg, total_items, maxlogM, ptrs);
    return;
  }
  const size_t smem = sizeof(cx<T>) * beta_czt_smem_elems(maxlogM, sizeof(T) == 8);
  dim3 grid(total_items), block(256);
  switch (kind) {
    case CZT_BETA_ANA: k_czt_beta_ana<T><<<grid, block, smem, st>>>(segs, nseg); break;
    case CZT_BETA_SYN: k_czt_beta_syn<T><<<grid, block, smem, st>>>(segs, nseg); break;
    case CZT_BETA_MW_DFT: k_beta_mw_dft<T><<<grid, block, smem, st>>>(segs, nseg); break;
    case CZT_BETA_RS: k_czt_beta_ana<T><<<grid, block, smem, st>>>(segs, nseg); break;
    case CZT_BETA_RS_FFT:
    case CZT_BETA_ANA_FFT: {  // persistent
      const size_t sm = beta_ana_fft_smem<T>(maxlogM);
      auto k = k_beta_ana_fft<T, 0>;
      if constexpr (sizeof(T) == sizeof(float)) {
        if (ulog == 11) k = k_beta_ana_fft<T, 11>;
        if (ulog == 12) k = k_beta_ana_fft<T, 12>;
        if (ulog == 13) k = k_beta_ana_fft<T, 13>;
      }
      const int g = std::min(total_items, alpha_czt_grid<T>(k, sm));
      k<<<g, block, sm, st>>>(segs, nseg, total_items, maxlogM);
      break;
    }
    case CZT_ALPHA_ANA_DIRECT:
      if constexpr (sizeof(T) == sizeof(float))
        launch_alpha_tc(false, segs, nseg, total_items, ptrs, st);  // tensor cores
      else
        k_alpha_ana_direct<T><<<grid, block, alpha_ana_direct_smem<T>(), st>>>(segs, nseg, ptrs);
      break;

    case CZT_BETA_ANA_DCT:
    case CZT_BETA_RS_DCT:
    case CZT_BETA_SYN_DCT: {  // persistent; uniform transform length: the specialised kernel
      const bool syn = kind == CZT_BETA_SYN_DCT;
      const size_t sm = beta_dct_smem<T>(syn);
      const int logN = (uniform_logM > 0) ? uniform_logM - 1 : 0;
      auto pick = [&](auto ana_k, auto syn_k) {
        if (syn) {
          const int g = std::min(total_items, alpha_czt_grid<T>(syn_k, sm));
          syn_k<<<g, block, sm, st>>>(segs, nseg, total_items);
        } else {
          const int g = std::min(total_items, alpha_czt_grid<T>(ana_k, sm));
          ana_k<<<g, block, sm, st>>>(segs, nseg, total_items);
        }
      };
      switch (logN) {
        case 11: pick(k_beta_ana_dct<T, 11>, k_beta_syn_dct<T, 11>); break;
        case 10: pick(k_beta_ana_dct<T, 10>, k_beta_syn_dct<T, 10>); break;
        case 9: pick(k_beta_ana_dct<T, 9>, k_beta_syn_dct<T, 9>); break;
        case 8: pick(k_beta_ana_dct<T, 8>, k_beta_syn_dct<T, 8>); break;
        default: pick(k_beta_ana_dct<T, 0>, k_beta_syn_dct<T, 0>); break;
      }
      break;
    }
    case CZT_BETA_SYN_FFT: {  // persistent
      const size_t sm = beta_syn_fft_smem<T>(maxlogM);
      auto k = k_beta_syn_fft<T, 0>;
      if constexpr (sizeof(T) == sizeof(float)) {
        if (ulog == 11) k = k_beta_syn_fft<T, 11>;
        if (ulog == 12) k = k_beta_syn_fft<T, 12>;
        if (ulog == 13) k = k_beta_syn_fft<T, 13>;
      }
      const int g = std::min(total_items, alpha_czt_grid<T>(k, sm));
      k<<<g, block, sm, st>>>(segs, nseg, total_items, maxlogM);
      break;
    }
    case CZT_ALPHA_SYN_DIRECT:
      if constexpr (sizeof(T) == sizeof(float))
        launch_alpha_tc(true, segs, nseg, total_items, ptrs, st);  // tensor cores
      else
        k_alpha_syn_direct<T><<<grid, block, alpha_syn_direct_smem<T>(1 << (maxlogM - 2)), st>>>(segs, nseg, ptrs);
      break;
    default: break;
  }
}

template <typename T>
cudaError_t czt_set_smem(int maxlogM) {
  // the chirp-z beta kernels (beta_czt_cols columns per CTA)
  const int smem = (int)(sizeof(cx<T>) * beta_czt_smem_elems(maxlogM, sizeof(T) == 8));
  cudaError_t e = cudaSuccess;
  e = cudaFuncSetAttribute(k_beta_mw_dft<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_czt_beta_ana<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  for (auto k : {k_czt_alpha_ana<T, false, 0>, k_czt_alpha_ana<T, true, 0>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)alpha_czt_smem<T>(maxlogM, false));
    if (e != cudaSuccess) return e;
  }
  e = cudaFuncSetAttribute(k_czt_alpha_syn<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)alpha_czt_smem<T>(maxlogM, true));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_beta_ana_fft<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)beta_ana_fft_smem<T>(maxlogM));
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(k_beta_syn_fft<T, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)beta_syn_fft_smem<T>(maxlogM));
  if (e != cudaSuccess) return e;
  if constexpr (sizeof(T) == sizeof(float)) {
    for (auto k : {k_czt_alpha_ana<T, false, 11>, k_czt_alpha_ana<T, false, 12>, k_czt_alpha_ana<T, false, 13>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)alpha_czt_smem<T>(maxlogM, false));
      if (e != cudaSuccess) return e;
    }
    for (auto k : {k_czt_alpha_syn<T, 11>, k_czt_alpha_syn<T, 12>, k_czt_alpha_syn<T, 13>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)alpha_czt_smem<T>(maxlogM, true));
      if (e != cudaSuccess) return e;
    }
    for (auto k : {k_beta_ana_fft<T, 11>, k_beta_ana_fft<T, 12>, k_beta_ana_fft<T, 13>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beta_ana_fft_smem<T>(maxlogM));
      if (e != cudaSuccess) return e;
    }
    for (auto k : {k_beta_syn_fft<T, 11>, k_beta_syn_fft<T, 12>, k_beta_syn_fft<T, 13>}) {
      e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beta_syn_fft_smem<T>(maxlogM));
      if (e != cudaSuccess) return e;
    }
  }
  for (auto k : {k_beta_ana_dct<T, 0>, k_beta_ana_dct<T, 8>, k_beta_ana_dct<T, 9>, k_beta_ana_dct<T, 10>,
                 k_beta_ana_dct<T, 11>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beta_dct_smem<T>(false));
    if (e != cudaSuccess) return e;
  }
  for (auto k : {k_beta_syn_dct<T, 0>, k_beta_syn_dct<T, 8>, k_beta_syn_dct<T, 9>, k_beta_syn_dct<T, 10>,
                 k_beta_syn_dct<T, 11>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)beta_dct_smem<T>(true));
    if (e != cudaSuccess) return e;
  }
  for (auto k : {k_czt_alpha_ana_seg<T, false>, k_czt_alpha_ana_seg<T, true>, k_czt_alpha_syn_seg<T, false>,
                 k_czt_alpha_syn_seg<T, true>}) {
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)alpha_seg_smem<T>());
    if (e != cudaSuccess) return e;
  }
  if constexpr (sizeof(T) == sizeof(double)) {  // FP32 plans take the tensor-core kernels
    e = cudaFuncSetAttribute(k_alpha_ana_direct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)alpha_ana_direct_smem<T>());
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_alpha_syn_direct<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)alpha_syn_direct_smem<T>(2048));
    if (e != cudaSuccess) return e;
  } else {
    e = alpha_tc_prepare();
    if (e != cudaSuccess) return e;
  }
  return cudaFuncSetAttribute(k_czt_beta_syn<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
}

}  // namespace s2dw
