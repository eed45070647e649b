// Instantiations of the chirp-z kernels for double.
#include "czt.cuh"

namespace s2dw {

template <>
void launch_czt<double>(int kind, const CztSeg<double>* segs, int nseg, int total_items, int maxlogM, const CallPtrs& ptrs,
                    cudaStream_t st, int uniform_logM) {
  launch_czt_impl<double>(kind, segs, nseg, total_items, maxlogM, ptrs, st, uniform_logM);
}

cudaError_t czt_prepare_f64(int maxlogM) { return czt_set_smem<double>(maxlogM); }

}  // namespace s2dw
