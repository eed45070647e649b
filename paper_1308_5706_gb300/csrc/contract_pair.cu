// Instantiations and launchers of the FP32 tile-pair contraction
// (contract_pair.cuh), and the per-call packing of f_lm into its layout.
#include "contract_pair.cuh"

namespace s2dw {

// fP[b][l][c] = f_{l, 32 b + c} for 32 b + c <= l < L, else 0 (Lrf rows per
// block).  Grid (ceil(Lrmax / 8), max blocks, jobs); 8 rows l per CTA.
__global__ void __launch_bounds__(256) k_fpack(const ContractDesc<float>* __restrict__ descs, CallPtrs ptrs) {
  const int job = blockIdx.z, b = blockIdx.y;
  const ContractDesc<float>* D = descs + job;
  const int L = D->L, Lrf = D->Lrf;
  if (32 * b >= L) return;
  const int l = blockIdx.x * 8 + (threadIdx.x >> 5), c = threadIdx.x & 31;
  if (l >= Lrf) return;
  const int m = 32 * b + c;
  const float2* __restrict__ f = reinterpret_cast<const float2*>(ptrs.f[job]);
  const float2 v = (l < L && m <= l) ? f[l * l + l + m] : make_float2(0.f, 0.f);
  const_cast<float2*>(D->fP)[((size_t)b * Lrf + l) * 32 + c] = v;
}

void launch_fpack(const ContractDesc<float>* descs, int njobs, int nbmax, int Lrmax, const CallPtrs& ptrs,
                  cudaStream_t st) {
  if (njobs <= 0 || nbmax <= 0) return;
  dim3 grid((Lrmax + 7) / 8, nbmax, njobs);
  k_fpack<<<grid, 256, 0, st>>>(descs, ptrs);
}

bool pair_two_tiles(int N) { return N <= 5; }

template <int N, int NSLOT, bool SYN, int HALVES, int MINB = 1>
static void pair_one(int ntasks, const ContractDesc<float>* descs, const PairTask* tasks, const CallPtrs& ptrs,
                     cudaStream_t st) {
  using G = PairGeom<N, NSLOT, SYN, HALVES>;
  k_contract_pair<N, NSLOT, SYN, HALVES, MINB><<<ntasks, 256 * HALVES, G::SMEM, st>>>(descs, tasks, ptrs);
}

template <int N, int NSLOT>
static void pair_dir(bool syn, int shape, int ntasks, const ContractDesc<float>* descs, const PairTask* tasks,
                     const CallPtrs& ptrs, cudaStream_t st) {
  if constexpr (N <= 5) {
    if (shape == kPairShapePair) {
      if (syn) pair_one<N, NSLOT, true, 2>(ntasks, descs, tasks, ptrs, st);
      else pair_one<N, NSLOT, false, 2>(ntasks, descs, tasks, ptrs, st);
      return;
    }
    if (shape == kPairShapeTile2) {
      if (syn) pair_one<N, NSLOT, true, 1, 2>(ntasks, descs, tasks, ptrs, st);
      else pair_one<N, NSLOT, false, 1, 2>(ntasks, descs, tasks, ptrs, st);
      return;
    }
  }
  if (syn) pair_one<N, NSLOT, true, 1>(ntasks, descs, tasks, ptrs, st);
  else pair_one<N, NSLOT, false, 1>(ntasks, descs, tasks, ptrs, st);
}

void launch_contract_pair(int N, int nslot, bool syn, int shape, const ContractDesc<float>* descs,
                          const PairTask* tasks, int ntasks, const CallPtrs& ptrs, cudaStream_t st) {
  if (ntasks <= 0) return;
  if (N == 1 && nslot == 1) {
    pair_dir<1, 1>(syn, shape, ntasks, descs, tasks, ptrs, st);
    return;
  }
  switch (N) {
    case 1: pair_dir<1, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 2: pair_dir<2, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 3: pair_dir<3, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 4: pair_dir<4, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 5: pair_dir<5, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 6: pair_dir<6, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 7: pair_dir<7, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    case 8: pair_dir<8, 2>(syn, shape, ntasks, descs, tasks, ptrs, st); break;
    default: break;
  }
}

template <int N, int NSLOT, int H, int MINB = 1>
static cudaError_t pair_attr_h() {
  cudaError_t e = cudaFuncSetAttribute(k_contract_pair<N, NSLOT, false, H, MINB>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PairGeom<N, NSLOT, false, H>::SMEM);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_contract_pair<N, NSLOT, true, H, MINB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PairGeom<N, NSLOT, true, H>::SMEM);
}
// every CTA shape: N <= 5 a pair of tiles, one tile, or one tile at two CTAs
// per SM; one tile above
template <int N, int NSLOT>
static cudaError_t pair_attr() {
  cudaError_t e = pair_attr_h<N, NSLOT, 1>();
  if (e != cudaSuccess) return e;
  if constexpr (N <= 5) {
    e = pair_attr_h<N, NSLOT, 2>();
    if (e != cudaSuccess) return e;
    e = pair_attr_h<N, NSLOT, 1, 2>();
  }
  return e;
}

// Shared-memory caps of every instantiation, once per device.
cudaError_t pair_prepare() {
  static unsigned long long dev_done = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 64 && (dev_done & (1ull << dev))) return cudaSuccess;
  cudaError_t (*fns[])() = {pair_attr<1, 1>, pair_attr<1, 2>, pair_attr<2, 2>, pair_attr<3, 2>, pair_attr<4, 2>,
                            pair_attr<5, 2>, pair_attr<6, 2>, pair_attr<7, 2>, pair_attr<8, 2>};
  for (auto f : fns) {
    e = f();
    if (e != cudaSuccess) return e;
  }
  if (dev < 64) dev_done |= 1ull << dev;
  return cudaSuccess;
}

cudaError_t pair_timeouts(int* count) {
  cudaError_t e = cudaMemcpyFromSymbol(count, g_pair_timeouts, sizeof(int));
  if (e != cudaSuccess) return e;
  const int zero = 0;
  return cudaMemcpyToSymbol(g_pair_timeouts, &zero, sizeof(int));
}

}  // namespace s2dw
