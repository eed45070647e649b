// tcgen05 building blocks (5th-generation tensor cores, sm_103a): TMEM
// allocation, shared-memory matrix descriptors, kind::tf32 matrix products
// with completion through an mbarrier (bounded waits), TMEM loads, and the
// split of an FP32 value into two TF32 parts.
//
// FP32 products from TF32 ones: x = hi(x) + lo(x) with hi = x rounded to TF32
// (10 explicit mantissa bits) and lo = x - hi rounded to TF32, so that
//   a b = hi(a) hi(b) + hi(a) lo(b) + lo(a) hi(b) + O(2^-21 |a b|);
// three MMAs accumulating in FP32 give FP32-level sums.  The tensor cores'
// FP32 accumulation loses up to about one unit in the last place of the
// accumulator per MMA (measured: the error grows with the number of MMAs
// accumulated), so the kernels issue all cross products (about 2^-11 of the
// sum) first, while the accumulator is still small, and the hi*hi products
// after them: the large sum then takes one truncation per K-step, as if the
// cross terms were kept apart.  Long sums are moved to registers chunk by
// chunk and added there with rounding to nearest.
#pragma once

#include <cstdint>

namespace s2dw {
namespace tc {

// Operand images in shared memory: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes (4 floats), each 128 contiguous bytes.  Core matrices
// adjacent along K are kLboF floats apart (32 + 4: the pad sends the four
// 4-float groups that a warp writes for one row's 32 consecutive k to
// distinct banks), 8-row groups (KC / 4) kLboF floats apart.
constexpr int kLboF = 36;

__host__ __device__ constexpr int img_off(int r, int k, int KC) {
  return (r >> 3) * (KC / 4) * kLboF + (k >> 2) * kLboF + (r & 7) * 4 + (k & 3);
}
// floats of an image of R rows (R % 8 == 0) and KC columns (KC % 8 == 0)
__host__ __device__ constexpr int img_floats(int R, int KC) { return (R / 8) * (KC / 4) * kLboF; }
// byte offset of the K-step s (8 TF32 columns = two core matrices) in an image
__host__ __device__ constexpr int img_kstep_bytes(int s) { return s * 2 * kLboF * 4; }

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (K-adjacent core matrices), stride-dimension byte offset (8-row
// groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, int KC) {
  const uint32_t lbo = kLboF * 4, sbo = (uint32_t)(KC / 4) * kLboF * 4;
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// Instruction descriptor, kind::tf32: D FP32, A and B TF32, both K-major,
// M x N (M = 128: N % 16 == 0, 16 <= N <= 256).
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// D[tmem] (+)= A B^T, issued by one thread.
__device__ __forceinline__ void mma_tf32(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_d),
      "l"(da), "l"(db), "r"(idesc), "r"(acc)
      : "memory");
}

// The mbarrier gets one arrival once every MMA this thread issued before has completed.
__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// The thread may be suspended in the wait (up to the hint, 0.1 ms) instead of
// spinning, so waiting warps do not take issue slots from working ones.
__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity), "r"(100000u)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.shared::cta.b64 st, [%0];\n}\n" ::"r"(mbar) : "memory");
}

// Wait for the phase of the given parity to complete; false after `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  while (!mbar_test(mbar, parity))
    if (clock64() - t0 > limit) return false;
  return true;
}

// about one second at the maximum SM clock
constexpr long long kWaitCycles = 2000000000LL;

// TMEM columns (power of two >= 32), allocated by one whole warp; the base
// address is written to *dst (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* dst, int ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)), "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_free(uint32_t taddr, int ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// generic-proxy shared-memory writes made visible to the tensor cores
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// TMEM loads, shape 32x32b: thread l of the warp gets lane (taddr lane) + l,
// consecutive 32-bit columns from (taddr column).  Loads and the wait are one
// asm statement, so the loaded registers cannot be read before the wait.
#define S2DW_R8(b) "=r"(r[b]), "=r"(r[b + 1]), "=r"(r[b + 2]), "=r"(r[b + 3]), "=r"(r[b + 4]), "=r"(r[b + 5]), \
                   "=r"(r[b + 6]), "=r"(r[b + 7])

// one load of 8 columns
__device__ __forceinline__ void tmem_ld8(uint32_t ta, float (&v)[8]) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : S2DW_R8(0)
      : "r"(ta)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) v[j] = __uint_as_float(r[j]);
}

// one load of 32 columns
__device__ __forceinline__ void tmem_ld32(uint32_t ta, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : S2DW_R8(0), S2DW_R8(8), S2DW_R8(16), S2DW_R8(24)
      : "r"(ta)
      : "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

// two loads of 8 columns (at ta and tb)
__device__ __forceinline__ void tmem_ld8x2(uint32_t ta, uint32_t tb, float (&va)[8], float (&vb)[8]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%16];\n"
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%17];\n"
      "tcgen05.wait::ld.sync.aligned;\n"
      : S2DW_R8(0), S2DW_R8(8)
      : "r"(ta), "r"(tb)
      : "memory");
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    va[j] = __uint_as_float(r[j]);
    vb[j] = __uint_as_float(r[8 + j]);
  }
}

#undef S2DW_R8

__device__ __forceinline__ float to_tf32(float x) {
  uint32_t h;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(x));
  return __uint_as_float(h);
}

__device__ __forceinline__ void split_tf32(float x, float& hi, float& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - hi);
}

}  // namespace tc
}  // namespace s2dw
