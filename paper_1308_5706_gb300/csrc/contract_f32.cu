// Instantiations of the contraction kernels for float (E = 4 rows per thread).
#include "contract.cuh"

namespace s2dw {

template <>
void launch_contract<float>(int N, int nslot, bool syn, const ContractDesc<float>* descs, const TileTask* tiles,
                         int ntiles, const CallPtrs& ptrs, cudaStream_t st) {
  launch_contract_impl<float, 4>(N, nslot, syn, descs, tiles, ntiles, ptrs, st);
}

template <>
void launch_syn_reduce<float>(const ReduceJobs& jobs, int njobs, int Lmax, cudaStream_t st) {
  if (njobs <= 0) return;
  dim3 grid((Lmax + 127) / 128, Lmax, njobs), block(128);
  k_syn_reduce<float><<<grid, block, 0, st>>>(jobs, 8 * 4);
}

int contract_rows_per_thread(bool fp64) { return fp64 ? 2 : 4; }

}  // namespace s2dw
