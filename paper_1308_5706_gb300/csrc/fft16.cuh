// Register-resident radix-16 FFT engine for one CTA of 256 threads.
//
// A power-of-two length M = 2^logM (5 <= logM <= 13) is split into stages of
// radix 16, 16, ..., R_last (R_last in {2, 4, 8, 16}).  Forward stages are
// decimation in frequency, in place: a block of size S = R*Q holding x[j+Q r]
// (r < R) becomes X[j+Q k] = (sum_r x[j+Q r] e^{-2 pi i rk/R}) e^{-2 pi i jk/S}.
// The output is in mixed-radix digit-reversed order, so a convolution needs
// the kernel spectrum in that same order (computed with the same stages) and
// an inverse that runs the stages backwards (decimation in time, conjugate
// twiddles, unnormalised: it returns M times the inverse DFT).
//
// The first forward stage reads its inputs through a functor and the last
// inverse stage hands its outputs to a functor, so inputs/outputs never pass
// through shared memory on the way in or out; the last forward stage, the
// pointwise product with the spectrum and the first inverse stage run on the
// same registers.  Shared memory holds M (+M/16 padding) complex values.
//
// Twiddle table (fft_twiddle_*): for each radix-16 level d = 0, 1, ... with
// block size S_d = M / 16^d and Q_d = S_d / 16, entries [k-1][j] =
// e^{-2 pi i j k / S_d} (k = 1..15, j < Q_d), levels stored one after the
// other; a butterfly's 15 twiddles are then coalesced loads across a warp.
#pragma once

#include "common.cuh"

namespace s2dw {

__host__ __device__ __forceinline__ int fpad(int v) { return v + (v >> 4); }
__host__ __device__ constexpr int fft_smem_elems(int M) { return M + (M >> 4); }

// e^{-2 pi i k/16}, k = 0..15 (cos, sin of multiples of pi/8)
template <typename T> __device__ __forceinline__ cx<T> w16(int k, bool inv) {
  const T c1 = (T)0.92387953251128675613, s1 = (T)0.38268343236508977173, h = (T)0.70710678118654752440;
  T re, im;
  switch (k & 15) {
    case 0: re = 1; im = 0; break;
    case 1: re = c1; im = -s1; break;
    case 2: re = h; im = -h; break;
    case 3: re = s1; im = -c1; break;
    case 4: re = 0; im = -1; break;
    case 5: re = -s1; im = -c1; break;
    case 6: re = -h; im = -h; break;
    case 7: re = -c1; im = -s1; break;
    case 8: re = -1; im = 0; break;
    case 9: re = -c1; im = s1; break;
    case 10: re = -h; im = h; break;
    case 11: re = -s1; im = c1; break;
    case 12: re = 0; im = 1; break;
    case 13: re = s1; im = c1; break;
    case 14: re = h; im = h; break;
    default: re = c1; im = s1; break;
  }
  return mkc<T>(re, inv ? -im : im);
}

template <typename T, bool INV>
__device__ __forceinline__ void dft2(cx<T>& a, cx<T>& b) {
  const cx<T> s = cadd<T>(a, b), d = csub<T>(a, b);
  a = s;
  b = d;
}

template <typename T, bool INV>
__device__ __forceinline__ void dft4(cx<T>& a0, cx<T>& a1, cx<T>& a2, cx<T>& a3) {
  if constexpr (sizeof(T) == 4) {
    // the six complex additions as packed f32x2 operations (one instruction
    // each instead of two); the +-i products stay scalar (they swap parts)
    const f2p p0 = pk2(a0.x, a0.y), p1 = pk2(a1.x, a1.y), p2 = pk2(a2.x, a2.y), p3 = pk2(a3.x, a3.y);
    const f2p s02 = add2(p0, p2), d02 = sub2(p0, p2), s13 = add2(p1, p3), d13 = sub2(p1, p3);
    upk2(add2(s02, s13), a0.x, a0.y);
    upk2(sub2(s02, s13), a2.x, a2.y);
    T dx, dy, ex, ey;
    upk2(d02, dx, dy);
    upk2(d13, ex, ey);
    if (!INV) {
      a1 = mkc<T>(dx + ey, dy - ex);  // d02 - i d13
      a3 = mkc<T>(dx - ey, dy + ex);  // d02 + i d13
    } else {
      a1 = mkc<T>(dx - ey, dy + ex);
      a3 = mkc<T>(dx + ey, dy - ex);
    }
    return;
  }
  const cx<T> s02 = cadd<T>(a0, a2), d02 = csub<T>(a0, a2);
  const cx<T> s13 = cadd<T>(a1, a3), d13 = csub<T>(a1, a3);
  a0 = cadd<T>(s02, s13);
  a2 = csub<T>(s02, s13);
  if (!INV) {
    a1 = mkc<T>(d02.x + d13.y, d02.y - d13.x);  // d02 - i d13
    a3 = mkc<T>(d02.x - d13.y, d02.y + d13.x);  // d02 + i d13
  } else {
    a1 = mkc<T>(d02.x - d13.y, d02.y + d13.x);
    a3 = mkc<T>(d02.x + d13.y, d02.y - d13.x);
  }
}

// In-register DFT of size R in natural order (X_k = sum_r v_r e^{-+2 pi i rk/R}).
template <typename T, int R, bool INV> struct DftR;
template <typename T, bool INV> struct DftR<T, 2, INV> {
  static __device__ __forceinline__ void run(cx<T> (&v)[2]) { dft2<T, INV>(v[0], v[1]); }
};
template <typename T, bool INV> struct DftR<T, 4, INV> {
  static __device__ __forceinline__ void run(cx<T> (&v)[4]) { dft4<T, INV>(v[0], v[1], v[2], v[3]); }
};
template <typename T, bool INV> struct DftR<T, 8, INV> {
  static __device__ __forceinline__ void run(cx<T> (&v)[8]) {
    // n = r + 2q (r < 2, q < 4), k = k1 + 4 k2
    dft4<T, INV>(v[0], v[2], v[4], v[6]);
    dft4<T, INV>(v[1], v[3], v[5], v[7]);
    // twiddle e^{-2 pi i r k1 / 8} = w16^{2 r k1}
#pragma unroll
    for (int k1 = 1; k1 < 4; ++k1) v[1 + 2 * k1] = cmul<T>(v[1 + 2 * k1], w16<T>(2 * k1, INV));
    cx<T> o[8];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cx<T> a = v[2 * k1], b = v[2 * k1 + 1];
      dft2<T, INV>(a, b);
      o[k1] = a;
      o[k1 + 4] = b;
    }
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = o[i];
  }
};
template <typename T, bool INV> struct DftR<T, 16, INV> {
  static __device__ __forceinline__ void run(cx<T> (&v)[16]) {
    // n = r + 4q, k = k1 + 4 k2: inner DFT4 over q, twiddle w16^{r k1}, outer DFT4 over r
#pragma unroll
    for (int r = 0; r < 4; ++r) dft4<T, INV>(v[r], v[r + 4], v[r + 8], v[r + 12]);
#pragma unroll
    for (int r = 1; r < 4; ++r)
#pragma unroll
      for (int k1 = 1; k1 < 4; ++k1) v[r + 4 * k1] = cmul<T>(v[r + 4 * k1], w16<T>(r * k1, INV));
    cx<T> o[16];
#pragma unroll
    for (int k1 = 0; k1 < 4; ++k1) {
      cx<T> a0 = v[4 * k1], a1 = v[4 * k1 + 1], a2 = v[4 * k1 + 2], a3 = v[4 * k1 + 3];
      dft4<T, INV>(a0, a1, a2, a3);
      o[k1] = a0;
      o[k1 + 4] = a1;
      o[k1 + 8] = a2;
      o[k1 + 12] = a3;
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = o[i];
  }
};

// Element offset of twiddle level d (block size M / 16^d) in the table.
__host__ __device__ __forceinline__ int fft_twiddle_level_offset(int logM, int d) {
  int off = 0;
  for (int i = 0; i < d; ++i) off += 15 * (1 << (logM - 4 * (i + 1)));
  return off;
}
// Entries of the whole table for length 2^logM (levels with twiddles only).
__host__ __device__ __forceinline__ int fft_twiddle_entries(int logM) {
  const int nlev = (logM & 3) ? (logM >> 2) : (logM >> 2) - 1;
  return fft_twiddle_level_offset(logM, nlev);
}

// Stages below work on NT transforms per CTA (buffers ST elements apart in
// shared memory): a thread loads its table values (twiddles, spectrum) once
// into registers and applies them to the NT transforms in turn, which
// divides the L1 table traffic by NT while only one transform's data is live.

// One in-place forward (DIF) stage of radix R on blocks of size S, smem -> smem.
// tw: this stage's twiddle level ([k-1][j], k < 16, j < Q; j = 0 entries are 1).
template <typename T, int R, int NT = 1>
__device__ __forceinline__ void fft_fwd_stage(cx<T>* A, int M, int S, const cx<T>* __restrict__ tw, int ST = 0) {
  const int Q = S / R;
  for (int u = threadIdx.x; u < M / R; u += blockDim.x) {
    const int j = u & (Q - 1), base = (u - j) * R + j;
    cx<T> w[R];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      cx<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = A[t * ST + fpad(base + Q * r)];
      DftR<T, R, false>::run(v);
#pragma unroll
      for (int k = 1; k < R; ++k) {
        if (t == 0) w[k] = ldk(tw + (k - 1) * Q + j);
        v[k] = cmul<T>(v[k], w[k]);
      }
#pragma unroll
      for (int k = 0; k < R; ++k) A[t * ST + fpad(base + Q * k)] = v[k];
    }
  }
}

// Inverse (DIT) of fft_fwd_stage, smem -> smem, unnormalised (x R).
template <typename T, int R, int NT = 1>
__device__ __forceinline__ void fft_inv_stage(cx<T>* A, int M, int S, const cx<T>* __restrict__ tw, int ST = 0) {
  const int Q = S / R;
  for (int u = threadIdx.x; u < M / R; u += blockDim.x) {
    const int j = u & (Q - 1), base = (u - j) * R + j;
    cx<T> w[R];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      cx<T> v[R];
#pragma unroll
      for (int k = 0; k < R; ++k) v[k] = A[t * ST + fpad(base + Q * k)];
#pragma unroll
      for (int k = 1; k < R; ++k) {
        if (t == 0) w[k] = ldk(tw + (k - 1) * Q + j);
        v[k] = cmulc<T>(v[k], w[k]);
      }
      DftR<T, R, true>::run(v);
#pragma unroll
      for (int r = 0; r < R; ++r) A[t * ST + fpad(base + Q * r)] = v[r];
    }
  }
}

// Innermost stage (Q = 1): forward DFT, product with the spectrum (entry k
// of block u stored at H[k (M/R) + u]), inverse DFT.  H == nullptr: forward
// only (used to build spectra).
template <typename T, int R, int NT = 1>
__device__ __forceinline__ void fft_mid_stage(cx<T>* A, int M, const cx<T>* __restrict__ H, T scale, int ST = 0) {
  for (int u = threadIdx.x; u < M / R; u += blockDim.x) {
    const int base = u * R;
    if (H) {
      cx<T> h[R];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = A[t * ST + fpad(base + r)];
        DftR<T, R, false>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) {
          if (t == 0) h[k] = ldk(H + k * (M / R) + u);
          v[k] = cmul<T>(v[k], h[k]);
        }
        DftR<T, R, true>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) A[t * ST + fpad(base + k)] = v[k];
      }
    } else {
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        cx<T> v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = A[t * ST + fpad(base + r)];
        DftR<T, R, false>::run(v);
#pragma unroll
        for (int k = 0; k < R; ++k) A[t * ST + fpad(base + k)] = cscale<T>(v[k], scale);
      }
    }
  }
}

template <typename T, int NT = 1>
__device__ __forceinline__ void fft_mid_dispatch(cx<T>* A, int M, int Rl, const cx<T>* H, T scale, int ST = 0) {
  switch (Rl) {
    case 2: fft_mid_stage<T, 2, NT>(A, M, H, scale, ST); break;
    case 4: fft_mid_stage<T, 4, NT>(A, M, H, scale, ST); break;
    case 8: fft_mid_stage<T, 8, NT>(A, M, H, scale, ST); break;
    default: fft_mid_stage<T, 16, NT>(A, M, H, scale, ST); break;
  }
}

// Radix schedule: logM = 4a + b; stages of 16 (a of them, the first fused with
// the input) then R_last = 2^b if b > 0, else the a-th radix-16 stage is the
// innermost one.  Returns the innermost radix and the number of smem-to-smem
// radix-16 stages between the first and the innermost.
__device__ __forceinline__ void fft_schedule(int logM, int& Rl, int& nmid16) {
  const int a = logM >> 2, b = logM & 3;
  if (b) {
    Rl = 1 << b;
    nmid16 = a - 1;
  } else {
    Rl = 16;
    nmid16 = a - 2;
  }
}

// Full convolution-by-FFT on one CTA:
//   A = DIT( DIF(input) .* H ),  input(v) supplies element v (natural order),
//   output(v, value) receives element v of M * (x conv h) for v < M.
// Requires logM >= 5.  Ends with a __syncthreads() only if WRITE_SMEM (the
// final values are then left in A, in natural order, with padding).
template <typename T, bool WRITE_SMEM, typename In, typename Out>
__device__ __forceinline__ void fft_convolve(cx<T>* A, int logM, const cx<T>* __restrict__ H,
                                             const cx<T>* __restrict__ tw, In input, Out output) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  // first forward stage (S = M), inputs from the functor
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = input(j + Q * r);
      DftR<T, 16, false>::run(v);
      if (j) {
#pragma unroll
        for (int k = 1; k < 16; ++k) v[k] = cmul<T>(v[k], ldk(tw + (k - 1) * Q + j));
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) A[fpad(j + Q * k)] = v[k];
    }
  }
  __syncthreads();
  int S = M / 16;
  for (int s = 0; s < nmid; ++s) {
    fft_fwd_stage<T, 16>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1));
    __syncthreads();
    S /= 16;
  }
  fft_mid_dispatch<T>(A, M, Rl, H, T(1));
  __syncthreads();
  for (int s = nmid - 1; s >= 0; --s) {
    S *= 16;
    fft_inv_stage<T, 16>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1));
    __syncthreads();
  }
  // last inverse stage (S = M), outputs to the functor (or back to smem)
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = A[fpad(j + Q * k)];
      if (j) {
#pragma unroll
        for (int k = 1; k < 16; ++k) v[k] = cmulc<T>(v[k], ldk(tw + (k - 1) * Q + j));
      }
      DftR<T, 16, true>::run(v);
      if (WRITE_SMEM) {
#pragma unroll
        for (int r = 0; r < 16; ++r) A[fpad(j + Q * r)] = v[r];
      } else {
#pragma unroll
        for (int r = 0; r < 16; ++r) output(j + Q * r, v[r]);
      }
    }
  }
  if (WRITE_SMEM) __syncthreads();
}

// Position in shared memory of frequency f after the forward stages: the
// digits of f in the radices (16, ..., 16, R_last), least significant first,
// weighted by the strides M/16, M/256, ..., 1 of the stages that produce them.
__device__ __forceinline__ int fft_pos(int f, int logM) {
  const int a = logM >> 2, b = logM & 3;
  int p = 0;
  for (int i = 0; i < a; ++i) p += ((f >> (4 * i)) & 15) << (logM - 4 * (i + 1));
  if (b) p += (f >> (4 * a)) & ((1 << b) - 1);
  return p;
}

// Innermost stage (Q = 1) alone, forward or inverse.
template <typename T, int R, bool INV>
__device__ __forceinline__ void fft_inner_stage(cx<T>* A, int M) {
  for (int u = threadIdx.x; u < M / R; u += blockDim.x) {
    const int base = u * R;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = A[fpad(base + r)];
    DftR<T, R, INV>::run(v);
#pragma unroll
    for (int k = 0; k < R; ++k) A[fpad(base + k)] = v[k];
  }
}

template <typename T, bool INV>
__device__ __forceinline__ void fft_inner_dispatch(cx<T>* A, int M, int Rl) {
  switch (Rl) {
    case 2: fft_inner_stage<T, 2, INV>(A, M); break;
    case 4: fft_inner_stage<T, 4, INV>(A, M); break;
    case 8: fft_inner_stage<T, 8, INV>(A, M); break;
    default: fft_inner_stage<T, 16, INV>(A, M); break;
  }
}

// Forward DFT F_f = sum_v x_v e^{-2 pi i f v/M} of input(v) (natural order),
// left in A with F_f at fpad(fft_pos(f)).  Ends with __syncthreads().
template <typename T, typename In>
__device__ __forceinline__ void fft_forward_from(cx<T>* A, int logM, const cx<T>* __restrict__ tw, In input) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> v[16];
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = input(j + Q * r);
      DftR<T, 16, false>::run(v);
      if (j) {
#pragma unroll
        for (int k = 1; k < 16; ++k) v[k] = cmul<T>(v[k], ldk(tw + (k - 1) * Q + j));
      }
#pragma unroll
      for (int k = 0; k < 16; ++k) A[fpad(j + Q * k)] = v[k];
    }
  }
  __syncthreads();
  int S = M / 16;
  for (int s = 0; s < nmid; ++s) {
    fft_fwd_stage<T, 16>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1));
    __syncthreads();
    S /= 16;
  }
  fft_inner_dispatch<T, false>(A, M, Rl);
  __syncthreads();
}

// Unnormalised inverse DFT x_v = sum_f F_f e^{+2 pi i f v/M} of a spectrum
// stored with F_f at fpad(fft_pos(f)); output(v, x_v) receives every v < M.
// Expects A complete (call after a __syncthreads()).
template <typename T, typename Out>
__device__ __forceinline__ void fft_inverse_to(cx<T>* A, int logM, const cx<T>* __restrict__ tw, Out output) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  fft_inner_dispatch<T, true>(A, M, Rl);
  __syncthreads();
  int S = M >> (4 * (nmid + 1));
  for (int s = nmid - 1; s >= 0; --s) {
    S *= 16;
    fft_inv_stage<T, 16>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1));
    __syncthreads();
  }
  const int Q = M / 16;
  for (int j = threadIdx.x; j < Q; j += blockDim.x) {
    cx<T> v[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) v[k] = A[fpad(j + Q * k)];
    if (j) {
#pragma unroll
      for (int k = 1; k < 16; ++k) v[k] = cmulc<T>(v[k], ldk(tw + (k - 1) * Q + j));
    }
    DftR<T, 16, true>::run(v);
#pragma unroll
    for (int r = 0; r < 16; ++r) output(j + Q * r, v[r]);
  }
}

// fft_convolve on NT transforms per CTA (buffers ST elements apart):
//   input(v, t, pre(v)) -> element v of transform t;
//   output(v, t, value, post(v)) consumes element v of transform t;
//   after_first() runs once all inputs have been read (after the first stage).
// IN_MASK / OUT_MASK: bit r clear means that the inputs v = j + r M/16 are
// zero (not read) / the outputs there are not needed (neither computed to
// the end nor passed on or stored): the chirp-z sums have inputs only in the
// first and last quarter and need outputs in one half of the period.
template <typename T, int NT, bool WRITE_SMEM, unsigned IN_MASK = 0xFFFFu, unsigned OUT_MASK = 0xFFFFu,
          typename Pre, typename In, typename Post, typename Out, typename AfterFirst>
__device__ __forceinline__ void fft_convolve_n(cx<T>* A, int ST, int logM, const cx<T>* __restrict__ H,
                                               const cx<T>* __restrict__ tw, Pre pre, In input, Post post,
                                               Out output, AfterFirst after_first) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> w[16];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        cx<T> v[16];
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = ((IN_MASK >> r) & 1u) ? input(j + Q * r, t, pre(j + Q * r)) : mkc<T>(0, 0);
        DftR<T, 16, false>::run(v);
#pragma unroll
        for (int k = 1; k < 16; ++k) {
          if (t == 0) w[k] = ldk(tw + (k - 1) * Q + j);
          v[k] = cmul<T>(v[k], w[k]);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) A[t * ST + fpad(j + Q * k)] = v[k];
      }
    }
  }
  __syncthreads();
  after_first();  // every input has been read: the caller may refill its input buffers
  int S = M / 16;
  for (int s = 0; s < nmid; ++s) {
    fft_fwd_stage<T, 16, NT>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1), ST);
    __syncthreads();
    S /= 16;
  }
  fft_mid_dispatch<T, NT>(A, M, Rl, H, T(1), ST);
  __syncthreads();
  for (int s = nmid - 1; s >= 0; --s) {
    S *= 16;
    fft_inv_stage<T, 16, NT>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1), ST);
    __syncthreads();
  }
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> w[16];
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        cx<T> v[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) v[k] = A[t * ST + fpad(j + Q * k)];
#pragma unroll
        for (int k = 1; k < 16; ++k) {
          if (t == 0) w[k] = ldk(tw + (k - 1) * Q + j);
          v[k] = cmulc<T>(v[k], w[k]);
        }
        DftR<T, 16, true>::run(v);
        if (WRITE_SMEM) {
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if ((OUT_MASK >> r) & 1u) A[t * ST + fpad(j + Q * r)] = v[r];
        } else {
#pragma unroll
          for (int r = 0; r < 16; ++r)
            if ((OUT_MASK >> r) & 1u) output(j + Q * r, t, v[r], post(j + Q * r));
        }
      }
    }
  }
  if (WRITE_SMEM) __syncthreads();
}

// ---- NT transforms per CTA (buffers ST elements apart) ----
template <typename T, int R, bool INV, int NT>
__device__ __forceinline__ void fft_inner_stage_n(cx<T>* A, int M, int ST) {
  for (int u = threadIdx.x; u < M / R; u += blockDim.x) {
    const int base = u * R;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      cx<T> v[R];
#pragma unroll
      for (int r = 0; r < R; ++r) v[r] = A[t * ST + fpad(base + r)];
      DftR<T, R, INV>::run(v);
#pragma unroll
      for (int k = 0; k < R; ++k) A[t * ST + fpad(base + k)] = v[k];
    }
  }
}

template <typename T, bool INV, int NT>
__device__ __forceinline__ void fft_inner_dispatch_n(cx<T>* A, int M, int Rl, int ST) {
  switch (Rl) {
    case 2: fft_inner_stage_n<T, 2, INV, NT>(A, M, ST); break;
    case 4: fft_inner_stage_n<T, 4, INV, NT>(A, M, ST); break;
    case 8: fft_inner_stage_n<T, 8, INV, NT>(A, M, ST); break;
    default: fft_inner_stage_n<T, 16, INV, NT>(A, M, ST); break;
  }
}

// fft_forward_from on NT transforms: input(v, x) fills x[t], t < NT, with
// element v of transform t.  after_input() runs once every input has been
// read (after the first stage's barrier).  Ends with __syncthreads().
// IN_MASK: bit r clear means that the inputs v = j + r M/16 are zero (not read).
template <typename T, int NT, unsigned IN_MASK = 0xFFFFu, typename In, typename AfterInput>
__device__ __forceinline__ void fft_forward_from_n(cx<T>* A, int ST, int logM, const cx<T>* __restrict__ tw,
                                                   In input, AfterInput after_input) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  {
    const int Q = M / 16;
    for (int j = threadIdx.x; j < Q; j += blockDim.x) {
      cx<T> v[NT][16];
#pragma unroll
      for (int r = 0; r < 16; ++r) {
        cx<T> x[NT];
        if ((IN_MASK >> r) & 1u) {
          input(j + Q * r, x);
        } else {
#pragma unroll
          for (int t = 0; t < NT; ++t) x[t] = mkc<T>(0, 0);
        }
#pragma unroll
        for (int t = 0; t < NT; ++t) v[t][r] = x[t];
      }
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        DftR<T, 16, false>::run(v[t]);
#pragma unroll
        for (int k = 1; k < 16; ++k) v[t][k] = cmul<T>(v[t][k], ldk(tw + (k - 1) * Q + j));
#pragma unroll
        for (int k = 0; k < 16; ++k) A[t * ST + fpad(j + Q * k)] = v[t][k];
      }
    }
  }
  __syncthreads();
  after_input();
  int S = M / 16;
  for (int s = 0; s < nmid; ++s) {
    fft_fwd_stage<T, 16, NT>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1), ST);
    __syncthreads();
    S /= 16;
  }
  fft_inner_dispatch_n<T, false, NT>(A, M, Rl, ST);
  __syncthreads();
}

// fft_inverse_to on NT transforms: output(v, y) receives element v of every
// transform (y[t]).  Expects A complete (call after a __syncthreads()).
// OUT_MASK: bit r clear means that the outputs v = j + r M/16 are not needed.
template <typename T, int NT, unsigned OUT_MASK = 0xFFFFu, typename Out>
__device__ __forceinline__ void fft_inverse_to_n(cx<T>* A, int ST, int logM, const cx<T>* __restrict__ tw,
                                                 Out output) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  fft_inner_dispatch_n<T, true, NT>(A, M, Rl, ST);
  __syncthreads();
  int S = M >> (4 * (nmid + 1));
  for (int s = nmid - 1; s >= 0; --s) {
    S *= 16;
    fft_inv_stage<T, 16, NT>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1), ST);
    __syncthreads();
  }
  const int Q = M / 16;
  for (int j = threadIdx.x; j < Q; j += blockDim.x) {
    cx<T> v[NT][16];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
#pragma unroll
      for (int k = 0; k < 16; ++k) v[t][k] = A[t * ST + fpad(j + Q * k)];
#pragma unroll
      for (int k = 1; k < 16; ++k) v[t][k] = cmulc<T>(v[t][k], ldk(tw + (k - 1) * Q + j));
      DftR<T, 16, true>::run(v[t]);
    }
#pragma unroll
    for (int r = 0; r < 16; ++r) {
      if (!((OUT_MASK >> r) & 1u)) continue;
      cx<T> y[NT];
#pragma unroll
      for (int t = 0; t < NT; ++t) y[t] = v[t][r];
      output(j + Q * r, y);
    }
  }
}

// ---------------------------------------------------------------------------
// Thread-group transforms: a CTA runs several transforms of length M side by
// side, each on its own group of nthr = M/16 threads (thread tid of the
// group) and its own shared-memory buffer, so that lengths below 4096 keep
// every thread busy.  The stage sequence is the one above (first radix-16
// stage, radix-16 stages, innermost R_last); callers put a __syncthreads()
// between stages (all groups run the same schedule).
// ---------------------------------------------------------------------------

// First forward stage fused with the input functor (in(v) gives element v).
template <typename T, typename In>
__device__ __forceinline__ void fftg_first_fwd(cx<T>* A, int M, int tid, const cx<T>* __restrict__ tw, In in) {
  const int Q = M / 16, j = tid;
  cx<T> v[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) v[r] = in(j + Q * r);
  DftR<T, 16, false>::run(v);
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmul<T>(v[k], ldk(tw + (k - 1) * Q + j));
#pragma unroll
  for (int k = 0; k < 16; ++k) A[fpad(j + Q * k)] = v[k];
}

// Radix-16 stage of block size S, forward (DIF) or inverse (DIT), smem -> smem.
template <typename T, bool INV>
__device__ __forceinline__ void fftg_stage16(cx<T>* A, int M, int S, int tid, int nthr, const cx<T>* __restrict__ tw) {
  const int Q = S / 16;
  for (int u = tid; u < M / 16; u += nthr) {
    const int j = u & (Q - 1), base = (u - j) * 16 + j;
    cx<T> v[16];
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = A[fpad(base + Q * r)];
    if (!INV) {
      DftR<T, 16, false>::run(v);
#pragma unroll
      for (int k = 1; k < 16; ++k) v[k] = cmul<T>(v[k], ldk(tw + (k - 1) * Q + j));
    } else {
#pragma unroll
      for (int k = 1; k < 16; ++k) v[k] = cmulc<T>(v[k], ldk(tw + (k - 1) * Q + j));
      DftR<T, 16, true>::run(v);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) A[fpad(base + Q * k)] = v[k];
  }
}

// Innermost stage (blocks of R consecutive entries), three forms:
//   MODE 0: forward DFT in place (Src == Dst);
//   MODE 1: Dst = inverse DFT of (Src .* H)   (spectrum entry k of block u at H[k (M/R) + u]);
//   MODE 2: Dst (+)= (forward DFT of Src) .* H   (accumulate unless first);
//   MODE 3: inverse DFT in place (Src == Dst).
template <typename T, int R, int MODE>
__device__ __forceinline__ void fftg_inner_r(const cx<T>* Src, cx<T>* Dst, int M, int tid, int nthr,
                                             const cx<T>* __restrict__ H, bool first) {
  for (int u = tid; u < M / R; u += nthr) {
    const int base = u * R;
    cx<T> v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = Src[fpad(base + r)];
    if (MODE == 1 || MODE == 3) {
      if (MODE == 1) {
#pragma unroll
        for (int k = 0; k < R; ++k) v[k] = cmul<T>(v[k], ldk(H + k * (M / R) + u));
      }
      DftR<T, R, true>::run(v);
#pragma unroll
      for (int k = 0; k < R; ++k) Dst[fpad(base + k)] = v[k];
    } else {
      DftR<T, R, false>::run(v);
      if (MODE == 0) {
#pragma unroll
        for (int k = 0; k < R; ++k) Dst[fpad(base + k)] = v[k];
      } else {
#pragma unroll
        for (int k = 0; k < R; ++k) {
          const cx<T> p = cmul<T>(v[k], ldk(H + k * (M / R) + u));
          Dst[fpad(base + k)] = first ? p : cadd<T>(Dst[fpad(base + k)], p);
        }
      }
    }
  }
}
template <typename T, int MODE>
__device__ __forceinline__ void fftg_inner(const cx<T>* Src, cx<T>* Dst, int M, int Rl, int tid, int nthr,
                                           const cx<T>* __restrict__ H, bool first = true) {
  switch (Rl) {
    case 2: fftg_inner_r<T, 2, MODE>(Src, Dst, M, tid, nthr, H, first); break;
    case 4: fftg_inner_r<T, 4, MODE>(Src, Dst, M, tid, nthr, H, first); break;
    case 8: fftg_inner_r<T, 8, MODE>(Src, Dst, M, tid, nthr, H, first); break;
    default: fftg_inner_r<T, 16, MODE>(Src, Dst, M, tid, nthr, H, first); break;
  }
}

// Last inverse stage fused with the output functor (out(v, value) for every v < M).
template <typename T, typename Out>
__device__ __forceinline__ void fftg_last_inv(const cx<T>* A, int M, int tid, const cx<T>* __restrict__ tw, Out out) {
  const int Q = M / 16, j = tid;
  cx<T> v[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) v[k] = A[fpad(j + Q * k)];
#pragma unroll
  for (int k = 1; k < 16; ++k) v[k] = cmulc<T>(v[k], ldk(tw + (k - 1) * Q + j));
  DftR<T, 16, true>::run(v);
#pragma unroll
  for (int r = 0; r < 16; ++r) out(j + Q * r, v[r]);
}

// Forward transform only (smem in natural order -> smem in the engine's
// order), values scaled by `scale`; used to build the kernel spectra.
template <typename T>
__device__ __forceinline__ void fft_forward_inplace(cx<T>* A, int logM, const cx<T>* __restrict__ tw, T scale) {
  const int M = 1 << logM;
  int Rl, nmid;
  fft_schedule(logM, Rl, nmid);
  fft_fwd_stage<T, 16>(A, M, M, tw);
  __syncthreads();
  int S = M / 16;
  for (int s = 0; s < nmid; ++s) {
    fft_fwd_stage<T, 16>(A, M, S, tw + fft_twiddle_level_offset(logM, s + 1));
    __syncthreads();
    S /= 16;
  }
  fft_mid_dispatch<T>(A, M, Rl, nullptr, scale);
  __syncthreads();
}

}  // namespace s2dw
