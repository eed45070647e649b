// Host launchers of the plan-time kernels (float64 unless stated).
#pragma once

#include "common.cuh"

namespace s2dw {

cudaError_t launch_kernel_values(double* kap, double* phi, double* sabs, double2* psi, double* q, int L, int N,
                                 int J, double lam, const double* glx, const double* glw, int Q, int P,
                                 double* I0, cudaStream_t st);
int twiddle_entries(int logM);  // entries of the FFT twiddle table of length 2^logM
cudaError_t launch_twiddles64(double2* tw, int logM, cudaStream_t st);  // that table (float64)
cudaError_t launch_mw_pre64(double2* pre, int L, cudaStream_t st);  // MW beta chirp, 2L-1 entries
// Segmented chirp-z tables (float64): twiddles of length 2^logM and the S
// analysis / synthesis kernel spectra (S x 2^logM each) of a band Lj.
cudaError_t launch_seg_build64(double2* tw, double2* Ha, double2* Hs, int L, int Lj, int logM, int P, int S,
                               cudaStream_t st);
cudaError_t launch_dh_weights(double* q, int L, cudaStream_t st);  // Eq. (18), 2L weights
// slabs l_first .. Lmax-1 (the edge arrays em/ee always cover l < Lmax)
cudaError_t launch_delta_build(double* d64, float* d32, double* em, int* ee, int Lmax, int l_first,
                               cudaStream_t st);
template <typename T>
cudaError_t launch_rtable(T* RS, const double* d64, const double* kap, const double* sabs, const int* slotj, int L,
                          int Lp, int N, int nslot, int kapL, cudaStream_t st);
cudaError_t launch_chirp_build64(double2* tw, double2* chirp_a, double2* pre_b, double2* post_b, double2* preS_b,
                                 double2* postS_b, double2* root_a, double2* bfft, double2* H, const double* q, int L,
                                 int logM,
                                 cudaStream_t st);
template <typename T>
cudaError_t launch_to_prec(cx<T>* dst, const double2* src, int64_t n, cudaStream_t st);
// n values of T in [-1/2, 1/2) from a hash of (seed, index): inputs for timing runs
template <typename T>
cudaError_t launch_fill_noise(T* dst, int64_t n, uint32_t seed, cudaStream_t st);

}  // namespace s2dw
