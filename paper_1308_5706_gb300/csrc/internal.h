// Internal descriptors shared by the plan, the launchers and the kernels.
#pragma once

#include "common.cuh"

namespace s2dw {

constexpr int MAXS = 66;   // wavelet scales (<= 64) plus headroom
constexpr int MAXB = 64;   // transforms per batched launch
constexpr int TILE = 32;   // contraction tile edge (m' and m)
constexpr int LCH = 8;     // l-chunk of the synthesis in-tile reduction

// One l-segment on which the scale held by each of the two accumulator
// slots is constant (slot s holds the scale j with j % 2 == s, or -1).
struct LSeg {
  int lo, hi;
  int j[2];
};

// Static, per-plan description of one contraction pass (wavelet scales with
// N orders, or the scaling function with N = 1), device resident.
template <typename T>
struct ContractDesc {
  const T* delta;    // Delta table (padded eighth domain), working precision
  // FP32 plans (tile-pair contraction, contract_pair.cuh):
  const float* dpair;  // Delta pair table of the plan's shared table
  const float* RSp;    // [nb][Lr][nslot][(N+1)/2][32]: R rows per 32-block of m', l outermost
  const cx<T>* fP;     // [nb][Lrf][32]: f_lm per 32-block of m (zero for m > l), packed per call
  int Lr, Lrf;         // l rows of RSp and fP (>= L + 7: a stage may read seven l past the last)
  const T* RS;       // [L][nslot][(N+1)/2][Lp]: Delta^l_{m',n_k} kappa^j(l) |s_{l,n_k}|, n_k >= 0
  cx<T>* P;          // synthesis partials [nbr][L][Lp32]
  int L, Lp, Lp32, nbr;
  int nseg;
  int N, nslot, eta_odd;   // eta_odd: N even -> eta = i
  int Lj[MAXS];            // per scale band-limit (support hi + 1)
  cx<T>* Y[MAXS];          // per scale cube [N][Lj][Lj] (analysis out / synthesis in)
  LSeg seg[2 * MAXS + 2];
};

// One tile pair of the FP32 contraction: blocks p <= q of 32 rows / columns;
// tile A = (m' block p, m block q), tile B = (q, p).  dbase: entry of the
// pair table holding l = lstart = 32 q (1024 entries per l follow).
struct PairTask {
  int prob;
  int p, q;
  int lstart, lend;
  int half;  // one-tile launches (N > 5): 0 = tile A, 1 = tile B
  long long dbase;
};

// l rows of padding after the tables the tile-pair contraction streams (the
// pair table's last run, the R rows and f values of each block): a pipeline
// stage of up to eight l may read seven l past a tile's last l; the values
// read there never enter the sums.
constexpr int kPairPadL = 8;

// Pair table of reach Lmax (a multiple of 32): pairs ordered by q, then p;
// the run of pair (p, q) holds Lmax - 32 q blocks of 32 x 32 entries.
// Entry of its first block (l = 32 q):
//   1024 * (Lmax q (q+1)/2 - 32 (q-1) q (q+1)/3 + p (Lmax - 32 q)).
__host__ __device__ __forceinline__ long long pair_run_base(int p, int q, int Lmax) {
  const long long Q = q;
  return 1024LL * ((long long)Lmax * Q * (Q + 1) / 2 - 32LL * (Q - 1) * Q * (Q + 1) / 3 + (long long)p * (Lmax - 32 * Q));
}
// entries of the whole table (+ one stage of read-ahead past the last run)
__host__ __device__ __forceinline__ long long pair_table_entries(int Lmax) {
  return pair_run_base(0, Lmax / 32, Lmax) + kPairPadL * 1024;
}

struct TileTask {
  int prob;    // index into the descriptor array of the launch
  int bmp;     // m' block
  int bm;      // m block
  int lstart;  // first l of the tile (max(32 bmp, 32 bm))
  int lend;    // last l with a nonzero contribution
};

// Per-call pointers, passed by value to the kernels.
struct CallPtrs {
  const void* f[MAXB];   // analysis input f_lm
  void* out[MAXB];       // synthesis output f_lm
  void* W[MAXB];         // wavelet coefficients
  void* Wphi[MAXB];      // scaling coefficients
};

enum CztKind {
  CZT_BETA_ANA = 0,
  CZT_ALPHA_ANA = 1,
  CZT_ALPHA_SYN = 2,
  CZT_BETA_SYN = 3,
  CZT_ALPHA_ANA_DIRECT = 4,  // small-band scales, direct sums
  CZT_ALPHA_SYN_DIRECT = 5,
  CZT_BETA_ANA_FFT = 6,      // beta sums as one FFT of length 4L (L a power of two)
  CZT_BETA_SYN_FFT = 7,
  CZT_ALPHA_ANA_SEG = 8,     // segmented chirp-z (bands small next to L)
  CZT_ALPHA_SYN_SEG = 9,
  CZT_BETA_MW_DFT = 10,      // MW grid, synthesis: torus coefficients from the L beta samples
  CZT_BETA_RS_FFT = 11,      // MW grid, synthesis: those coefficients evaluated on the DH beta grid
  CZT_BETA_RS = 12,          //   (single FFT, or chirp-z for non-power-of-two L)
  CZT_BETA_ANA_DCT = 13,     // beta sums as half-length transforms (L a power of two, L >= 16)
  CZT_BETA_SYN_DCT = 14,
  CZT_BETA_RS_DCT = 15       //   (MW grid, synthesis: evaluation on the DH beta grid)
};
// Or-ed into an alpha chirp-z kind: the list may hold segments with an odd row
// count N nb (MW grid), whose last row pair has one row.
constexpr int CZT_ODD_ROWS = 0x100;
// shared memory of the segmented chirp-z kernels: two buffers of M' (+ padding)
// for each of the 4096 / M' row pairs of a CTA
template <typename T>
constexpr size_t alpha_seg_smem() { return 2 * (size_t)(4096 + 4096 / 16) * 2 * sizeof(T); }
constexpr int kDirectMaxLj = 32;     // synthesis: direct alpha sums for L_j <= 32
constexpr int kDirectMaxLjAna = 32;  // analysis: direct (matrix-product) alpha sums for L_j <= 32
// tile of the direct analysis kernel: samples per CTA, rows per pass, rows per CTA
constexpr int kAgCols = 128, kAgRows = 64, kAgChunk = 512;
template <typename T>  // B tile + A tile (FP32 stores each A value twice)
constexpr size_t alpha_ana_direct_smem() {
  return (size_t)(2 * kDirectMaxLjAna - 1) * (kAgCols + kAgRows * (sizeof(T) == 4 ? 2 : 1)) * sizeof(T);
}
// row pairs (complex transforms) per CTA of the alpha chirp-z kernels: one
// (FP32 measured 9% faster at three CTAs per SM than two transforms per CTA
// sharing their table loads at two CTAs per SM; FP64 buffers allow one)
__host__ __device__ constexpr int alpha_czt_nt(bool fp64) { return (void)fp64, 1; }
// adjacent columns per CTA of the single-FFT beta kernels (FP32: a 16-byte pair)
__host__ __device__ constexpr int beta_fft_nt(bool fp64) { return fp64 ? 1 : 2; }
// adjacent columns per CTA of the chirp-z beta kernels for transforms of
// length 2^logM: FP32 a 16-byte pair up to 2^12, one at 2^13 (so that a CTA's
// buffers stay at 2 x 4352 complex); FP64 one
__host__ __device__ constexpr int beta_czt_cols(int logM, bool fp64) { return (fp64 || logM >= 13) ? 1 : 2; }
inline int direct_rows_syn(bool fp64) { return fp64 ? 4 : 8; }  // 32-byte line per alpha sample

// One segment of a chirp-z launch: all columns / row pairs of one scale of
// one transform.
template <typename T>
struct CztSeg {
  int start;      // first CTA index of this segment
  int items;
  int job;        // index into CallPtrs
  int L, Lj, N, logM;
  int64_t woff;   // element offset of this scale in W (or 0 for Wphi)
  int is_phi;     // 1: W pointer is CallPtrs::Wphi
  cx<T>* buf_in;  // plan workspace input (X / Y buffers)
  cx<T>* buf_out; // plan workspace output
  const cx<T>* H; // bit-reversed chirp kernel spectrum, scaled by 1/M
  const cx<T>* tw;
  const cx<T>* pre;
  const cx<T>* post;
  T scale;
  int P, nsegs;   // segmented chirp-z: samples per segment, segments
  int nb;         // beta samples per gamma sample (rows of X, V and W per g): 2L, or L on the MW grid
};

// Direct alpha sums on the tensor cores (FP32 plans, scales with L_j <= 32;
// alpha_tc.cu).  Basis tables: one per scale and direction, built per plan.
size_t alpha_tc_table_floats(int L, int Lj, bool syn);
cudaError_t alpha_tc_build_table(float* out, int L, int Lj, bool syn, cudaStream_t st);
int alpha_tc_items(int L, int rows, bool syn);
void launch_alpha_tc(bool syn, const CztSeg<float>* segs, int nseg, int total_items, const CallPtrs& ptrs,
                     cudaStream_t st);
cudaError_t alpha_tc_prepare();
cudaError_t alpha_tc_timeouts(int* count);  // reads and resets the device count
cudaError_t alpha_tc_wait_probe(long long limit, cudaStream_t st);  // a wait that runs out

// Per-job parameters of the batched final synthesis reduction.
struct ReduceJobs {
  const void* dw[MAXB];
  const void* dp[MAXB];
  void* out[MAXB];
  int L[MAXB];
  int lend[MAXB];
  int Lphi[MAXB];
  int sht[MAXB];  // 1: forward spherical harmonic transform (factor 1/(2 pi), see s2dw_sht_forward)
};

template <typename T>
void launch_contract(int N, int nslot, bool syn, const ContractDesc<T>* descs, const TileTask* tiles,
                     int ntiles, const CallPtrs& ptrs, cudaStream_t st);
// FP32 tile-pair contraction and its tables (contract_pair.cu)
bool pair_two_tiles(int N);  // a CTA may compute both tiles of a pair (N <= 5)
// CTA shapes of the FP32 contraction: the tasks name pairs and each CTA
// computes both tiles (N <= 5 only), or each task names one tile (its half),
// at one CTA per SM (the only shape for N > 5) or at two (N <= 5, 128
// registers per thread)
constexpr int kPairShapePair = 0, kPairShapeTile = 1, kPairShapeTile2 = 2;
void launch_contract_pair(int N, int nslot, bool syn, int shape, const ContractDesc<float>* descs,
                          const PairTask* tasks, int ntasks, const CallPtrs& ptrs, cudaStream_t st);
void launch_fpack(const ContractDesc<float>* descs, int njobs, int nbmax, int Lrmax, const CallPtrs& ptrs,
                  cudaStream_t st);
cudaError_t launch_pair_table(float* out, const double* d64, int Lmax, cudaStream_t st);
cudaError_t launch_rtable_pair(float* RSp, const double* d64, const double* kap, const double* sabs,
                               const int* slotj, int L, int Lr, int N, int nslot, int kapL, cudaStream_t st);
cudaError_t pair_prepare();
cudaError_t pair_timeouts(int* count);  // reads and resets the device count
template <typename T>
void launch_czt(int kind, const CztSeg<T>* segs, int nseg, int total_items, int maxlogM,
                const CallPtrs& ptrs, cudaStream_t st, int uniform_logM);
template <typename T>
void launch_syn_reduce(const ReduceJobs& jobs, int njobs, int Lmax, cudaStream_t st);

template <> void launch_contract<float>(int, int, bool, const ContractDesc<float>*, const TileTask*, int,
                                        const CallPtrs&, cudaStream_t);
template <> void launch_contract<double>(int, int, bool, const ContractDesc<double>*, const TileTask*, int,
                                         const CallPtrs&, cudaStream_t);
template <> void launch_czt<float>(int, const CztSeg<float>*, int, int, int, const CallPtrs&, cudaStream_t, int);
template <> void launch_czt<double>(int, const CztSeg<double>*, int, int, int, const CallPtrs&, cudaStream_t, int);
template <> void launch_syn_reduce<float>(const ReduceJobs&, int, int, cudaStream_t);
template <> void launch_syn_reduce<double>(const ReduceJobs&, int, int, cudaStream_t);
cudaError_t czt_prepare_f32(int maxlogM);
cudaError_t czt_prepare_f64(int maxlogM);
int contract_rows_per_thread(bool fp64);
constexpr int kDeltaPad = 64;     // spare entries after a Delta table (row-segment copies)
constexpr int kDeltaFront = 512;  // zero entries before it: the contraction's unguarded row
                                  // copies start up to 324 entries early (small l)

}  // namespace s2dw
