// Instantiations of the contraction kernels for double (E = 2 rows per thread).
#include "contract.cuh"

namespace s2dw {

template <>
void launch_contract<double>(int N, int nslot, bool syn, const ContractDesc<double>* descs, const TileTask* tiles,
                         int ntiles, const CallPtrs& ptrs, cudaStream_t st) {
  launch_contract_impl<double, 2>(N, nslot, syn, descs, tiles, ntiles, ptrs, st);
}

template <>
void launch_syn_reduce<double>(const ReduceJobs& jobs, int njobs, int Lmax, cudaStream_t st) {
  if (njobs <= 0) return;
  dim3 grid((Lmax + 127) / 128, Lmax, njobs), block(128);
  k_syn_reduce<double><<<grid, block, 0, st>>>(jobs, 8 * 2);
}

}  // namespace s2dw
