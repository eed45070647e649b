// Shared device helpers for the sm_103a wavelet transform kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace s2dw {

template <typename T> struct CxT;
template <> struct CxT<float> { typedef float2 type; };
template <> struct CxT<double> { typedef double2 type; };
template <typename T> using cx = typename CxT<T>::type;

template <typename T> __host__ __device__ __forceinline__ cx<T> mkc(T x, T y) {
  cx<T> r;
  r.x = x;
  r.y = y;
  return r;
}
template <typename T> __device__ __forceinline__ cx<T> cadd(cx<T> a, cx<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ cx<T> csub(cx<T> a, cx<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ cx<T> cmul(cx<T> a, cx<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ cx<T> cmulc(cx<T> a, cx<T> b) {  // a * conj(b)
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T> __device__ __forceinline__ cx<T> cconj(cx<T> a) { return mkc<T>(a.x, -a.y); }
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
// a * i^k
template <typename T> __device__ __forceinline__ cx<T> cmul_ipow(cx<T> a, int k) {
  switch (k & 3) {
    case 0: return a;
    case 1: return mkc<T>(-a.y, a.x);
    case 2: return mkc<T>(-a.x, -a.y);
    default: return mkc<T>(a.y, -a.x);
  }
}

// Padded eighth-domain layout of the Delta table (Delta^l_{m'm} = d^l_{m'm}(pi/2)).
// Slab l holds c = floor(l/4)+1 groups of 4 rows; rows 4q..4q+3 store columns
// 4q .. 4c-1 (zero beyond l), so every entry with m >= 4*floor(m'/4) is present
// and 4 consecutive columns starting at a multiple of 4 are 16-byte aligned.
__host__ __device__ __forceinline__ int64_t delta_slab_offset(int l) {
  int64_t C = l >> 2, c = C + 1, r = l & 3;
  return (32 * C * (C + 1) * (C + 2)) / 3 + r * 8 * c * (c + 1);
}
__host__ __device__ __forceinline__ int64_t delta_slab_size(int l) {
  int64_t c = (l >> 2) + 1;
  return 8 * c * (c + 1);
}
// Offset of entry (m', m) inside slab l (requires m >= 4*floor(m'/4)).
__host__ __device__ __forceinline__ int delta_entry(int l, int mp, int m) {
  int c = (l >> 2) + 1, q = mp >> 2, r = mp & 3;
  return 16 * q * c - 8 * q * (q - 1) + r * 4 * (c - q) + (m - 4 * q);
}
// Entry index = slab_offset + B*c + A with per-row constants (used in hot loops):
//   A(m', m) = -8q(q-1) - 4rq + m - 4q,  B(m') = 16q + 4r.
__host__ __device__ __forceinline__ int delta_row_A(int mp, int m) {
  int q = mp >> 2, r = mp & 3;
  return -8 * q * (q - 1) - 4 * r * q + m - 4 * q;
}
__host__ __device__ __forceinline__ int delta_row_B(int mp) { return 16 * (mp >> 2) + 4 * (mp & 3); }

static inline int64_t delta_table_entries(int Lmax) { return delta_slab_offset(Lmax); }


// cp.async (Ampere-style asynchronous global -> shared copies)
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
// 16 bytes to a 32-bit shared-memory address: whole (no size operand) or
// the first src_bytes with the rest zero-filled
__device__ __forceinline__ void cp_async16_s(uint32_t saddr, const void* gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_s(uint32_t saddr, const void* gmem, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(saddr), "l"(gmem), "r"(src_bytes) : "memory");
}
// one element of 4, 8 or 16 bytes, cached in L1 (.ca allows the small sizes)
template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void* smem, const void* gmem) {
  const unsigned s = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
// Asks L2 to fetch the 16-byte aligned part of [p, p + bytes) ahead of use
// (the bytes must lie inside one allocation; the hint never faults on them).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes) {
  const uintptr_t a = ((uintptr_t)p + 15) & ~(uintptr_t)15, e = ((uintptr_t)p + bytes) & ~(uintptr_t)15;
  if (e > a) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(a), "r"((uint32_t)(e - a)) : "memory");
}

// Read-only table loads (twiddles, chirps, kernel spectra) marked to be
// evicted last from L1, so that the single-use rows streaming past them do
// not push them out.
__device__ __forceinline__ float2 ldk(const float2* p) {
  float2 r;
  asm("ld.global.nc.L1::evict_last.v2.f32 {%0, %1}, [%2];" : "=f"(r.x), "=f"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ double2 ldk(const double2* p) {
  double2 r;
  asm("ld.global.nc.L1::evict_last.v2.f64 {%0, %1}, [%2];" : "=d"(r.x), "=d"(r.y) : "l"(p));
  return r;
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }


// Packed float pairs (two FP32 lanes per 64-bit register) for the sm_100+
// f32x2 instructions: one instruction per two multiply-adds.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p pk2(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(f2p v, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2p fma2(f2p a, f2p b, f2p c) {
  f2p d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ f2p add2(f2p a, f2p b) {
  f2p d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p sub2(f2p a, f2p b) {
  f2p d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ f2p mul2(f2p a, f2p b) {
  f2p d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

}  // namespace s2dw
