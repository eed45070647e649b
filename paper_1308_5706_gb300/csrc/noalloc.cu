// Delta-table builder that allocates no device memory.
//
// The regular plan path builds the Wigner Delta table with a temporary
// cudaMalloc'd edge table (mantissa + exponent of Delta^l_{l,m}).  Here that
// scratch lives in one file-scope __device__ array instead, sized for band
// limits up to kNoAllocMaxL; the caller provides the output table.
#include <mutex>

#include "../../include/s2dw.h"
#include "plan_kernels.h"

namespace {

constexpr int kNoAllocMaxL = 1024;
constexpr size_t kEdgeEntries = (size_t)kNoAllocMaxL * (kNoAllocMaxL + 1) / 2;
constexpr size_t kScratchBytes = kEdgeEntries * (sizeof(double) + sizeof(int));  // 6.3 MB

// Edge table scratch: kEdgeEntries doubles (mantissas), then kEdgeEntries ints
// (binary exponents).  Every device that loads the library holds it until exit.
static __device__ __align__(256) unsigned char g_delta_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once
// per device; host code must not use the symbol's host-side stand-in).
int scratch_for_current_device(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return S2DW_ECUDA;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_delta_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return S2DW_ECUDA;
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return S2DW_OK;
}

}  // namespace

extern "C" int s2dw_delta_table_noalloc(int Lmax, double* table64, float* table32, int64_t* entries,
                                        void* stream) {
  if (Lmax < 1) return S2DW_EINVAL;
  if (Lmax > kNoAllocMaxL) return S2DW_ENOTSUP;
  const int64_t n = s2dw::delta_table_entries(Lmax);
  if (entries) *entries = n;
  if (!table64) return table32 ? S2DW_EINVAL : S2DW_OK;
  void* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != S2DW_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  double* em = reinterpret_cast<double*>(scratch);
  int* ee = reinterpret_cast<int*>(reinterpret_cast<unsigned char*>(scratch) + kEdgeEntries * sizeof(double));
  // padded entries of the output must be zero; every edge entry used is rewritten
  if (cudaMemsetAsync(table64, 0, (size_t)n * sizeof(double), st) != cudaSuccess) return S2DW_ECUDA;
  if (table32 && cudaMemsetAsync(table32, 0, (size_t)n * sizeof(float), st) != cudaSuccess) return S2DW_ECUDA;
  if (s2dw::launch_delta_build(table64, table32, em, ee, Lmax, 0, st) != cudaSuccess) return S2DW_ECUDA;
  return S2DW_OK;
}
