// Instantiations of the chirp-z kernels for float.
#include "czt.cuh"

namespace s2dw {

template <>
void launch_czt<float>(int kind, const CztSeg<float>* segs, int nseg, int total_items, int maxlogM, const CallPtrs& ptrs,
                    cudaStream_t st, int uniform_logM) {
  launch_czt_impl<float>(kind, segs, nseg, total_items, maxlogM, ptrs, st, uniform_logM);
}

cudaError_t czt_prepare_f32(int maxlogM) { return czt_set_smem<float>(maxlogM); }

}  // namespace s2dw
