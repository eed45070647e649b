// C ABI: plans, the shared Delta table, launch lists, analysis and synthesis.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/s2dw.h"
#include "internal.h"
#include "plan_kernels.h"
#include "steer.h"

using namespace s2dw;

namespace {

inline int round_up(int x, int a) { return (x + a - 1) / a * a; }
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct CudaFail {
  cudaError_t err;
};
inline void ck(cudaError_t e) {
  if (e != cudaSuccess) throw CudaFail{e};
}

// Segmented chirp-z choice for a band Lj on a grid of band L whose chirp-z
// length is 2^logM: the length M' = 2^logMs (512 <= M' <= min(M/2, 4096)) and
// S = ceil(n / P) segments of P = M' - 2 Lj + 2 samples (n = 2L - 1) that
// minimise the FFT work (S + 1) M' log2 M', used where that is below 0.85 of
// the two FFTs of length M of one convolution (else S = 0).
void seg_choice(int L, int Lj, int logM, int& logMs, int& P, int& S) {
  const int n = 2 * L - 1;
  double best = 0.85 * 2.0 * (double)(1 << logM) * logM;
  logMs = P = S = 0;
  for (int lm = 9; lm <= std::min(logM - 1, 12); ++lm) {
    const int Mp = 1 << lm, p = Mp - 2 * Lj + 2;
    if (p <= 0) continue;
    const int s = (n + p - 1) / p;
    if (s > 64) continue;
    const double c = (double)(s + 1) * Mp * lm;
    if (c < best) {
      best = c;
      logMs = lm;
      P = p;
      S = s;
    }
  }
}

// J_max = ceil(log_lam L) by an integer loop (Sec. 2.2); -1 when it exceeds
// kJmaxCap (lambda so close to 1 that the loop would not end in reasonable
// time; such a plan would exceed the 64-scale limit anyway unless J0 were huge).
constexpr int kJmaxCap = 1 << 20;
int jmax_of(int L, double lam) {
  int J = 0;
  double p = 1.0;
  while (p < L) {
    p *= lam;
    if (++J > kJmaxCap) return -1;
  }
  return J;
}

// Gauss-Legendre nodes/weights on [-1, 1] (Newton iteration on P_Q).
void gauss_legendre(int Q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(Q, 0.0);
  w.assign(Q, 0.0);
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < Q; ++i) {
    double z = std::cos(pi * (i + 0.75) / (Q + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= Q; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = Q * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = z;
    w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Library-wide non-blocking stream for set-up copies and frees, and the
// device's stream-ordered memory pool configured to keep freed memory cached:
// creating and destroying plans then never synchronises the whole device
// (plain cudaFree / cudaMemcpy on the legacy stream would drain every stream
// of a serving process).
std::mutex g_setup_mu;
cudaStream_t g_setup_stream[64] = {};

// Kernel attributes (shared-memory limits sized for every plan, L <= 2048)
// are set once per device and precision under a lock, so that creating a plan
// in one host thread never changes an attribute of a kernel that another
// thread is launching.
std::mutex g_prep_mu;
void kernels_prepare(bool fp64, bool pair) {
  int dev = 0;
  ck(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) throw CudaFail{cudaErrorInvalidDevice};
  static unsigned long long done_czt[2] = {0, 0}, done_pair = 0;
  const unsigned long long bit = 1ull << dev;
  std::lock_guard<std::mutex> lk(g_prep_mu);
  if (!(done_czt[fp64 ? 1 : 0] & bit)) {
    ck(fp64 ? czt_prepare_f64(13) : czt_prepare_f32(13));
    done_czt[fp64 ? 1 : 0] |= bit;
  }
  if (pair && !(done_pair & bit)) {
    ck(pair_prepare());
    done_pair |= bit;
  }
}
cudaStream_t setup_stream() {
  int dev = 0;
  ck(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_setup_mu);
  if (dev < 0 || dev >= 64) throw CudaFail{cudaErrorInvalidDevice};
  if (!g_setup_stream[dev]) {
    ck(cudaStreamCreateWithFlags(&g_setup_stream[dev], cudaStreamNonBlocking));
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      uint64_t thr = 16ull << 30;  // keep up to 16 GiB of freed blocks cached
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  return g_setup_stream[dev];
}
template <typename P>
void amalloc(P** p, size_t bytes, cudaStream_t st) {
  ck(cudaMallocAsync(reinterpret_cast<void**>(p), bytes, st));
}
inline void afree(void* p, cudaStream_t st) {
  if (p) cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------------------
// Process-wide Delta tables, reference counted (one per band-limit reach).
// ---------------------------------------------------------------------------
struct DeltaTab {
  int Lmax;
  int device;
  double* d64;  // entry 0 of the table (kDeltaFront zero entries precede it)
  float* d32;
  int refs;
  size_t bytes;
  double* raw64 = nullptr;  // the allocations
  float* raw32 = nullptr;
  float* pair32 = nullptr;  // pair table of the FP32 tile-pair contraction (built for the first FP32 plan)
};
std::mutex g_mu;
std::vector<DeltaTab*> g_tabs;

DeltaTab* delta_acquire(int L, cudaStream_t st) {
  int dev = 0;
  ck(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_mu);
  DeltaTab* best = nullptr;
  for (DeltaTab* t : g_tabs)
    if (t->device == dev && t->Lmax >= L && (!best || t->Lmax < best->Lmax)) best = t;
  if (best) {
    best->refs++;
    return best;
  }
  // Size classes (multiples of 64 up to 256, then of 256) keep the number of
  // distinct tables small when plans of many band-limits come and go.  Slab l
  // does not depend on Lmax, so the slabs of the largest existing table are
  // copied and only the new ones are computed.
  const int Lmax = L <= 256 ? round_up(L, 64) : round_up(L, 256);
  DeltaTab* donor = nullptr;
  for (DeltaTab* u : g_tabs)
    if (u->device == dev && u->Lmax < Lmax && (!donor || u->Lmax > donor->Lmax)) donor = u;
  const int l_first = donor ? donor->Lmax : 0;
  const int64_t entries = delta_table_entries(Lmax) + 64;  // + read-ahead pad
  DeltaTab* t = new DeltaTab{Lmax, dev, nullptr, nullptr, 1, 0};
  double* em = nullptr;
  int* ee = nullptr;
  try {
    // kDeltaPad spare entries: the contraction copies 16-byte chunks of row
    // segments that may run past the last row of the last slab
    amalloc(&t->raw64, (kDeltaFront + entries + kDeltaPad) * sizeof(double), st);
    amalloc(&t->raw32, (kDeltaFront + entries + kDeltaPad) * sizeof(float), st);
    ck(cudaMemsetAsync(t->raw64, 0, kDeltaFront * sizeof(double), st));
    ck(cudaMemsetAsync(t->raw32, 0, kDeltaFront * sizeof(float), st));
    t->d64 = t->raw64 + kDeltaFront;
    t->d32 = t->raw32 + kDeltaFront;
    t->bytes = entries * (sizeof(double) + sizeof(float));
    const int64_t kept = delta_slab_offset(l_first);
    if (donor) {
      ck(cudaMemcpyAsync(t->d64, donor->d64, kept * sizeof(double), cudaMemcpyDeviceToDevice, st));
      ck(cudaMemcpyAsync(t->d32, donor->d32, kept * sizeof(float), cudaMemcpyDeviceToDevice, st));
    }
    ck(cudaMemsetAsync(t->d64 + kept, 0, (entries + kDeltaPad - kept) * sizeof(double), st));
    ck(cudaMemsetAsync(t->d32 + kept, 0, (entries + kDeltaPad - kept) * sizeof(float), st));
    const size_t ne = (size_t)Lmax * (Lmax + 1) / 2;
    amalloc(&em, ne * sizeof(double), st);
    amalloc(&ee, ne * sizeof(int), st);
    ck(launch_delta_build(t->d64, t->d32, em, ee, Lmax, l_first, st));
    afree(em, st);
    afree(ee, st);
    ck(cudaStreamSynchronize(st));
  } catch (...) {
    cudaStreamSynchronize(st);
    afree(em, st);
    afree(ee, st);
    afree(t->raw64, st);
    afree(t->raw32, st);
    delete t;
    throw;
  }
  g_tabs.push_back(t);
  return t;
}

// The FP32 pair table of a shared table (built from its FP64 slabs on first need).
void delta_pair_ensure(DeltaTab* t, cudaStream_t st) {
  std::lock_guard<std::mutex> lk(g_mu);
  if (t->pair32) return;
  float* pt = nullptr;
  amalloc(&pt, (size_t)pair_table_entries(t->Lmax) * sizeof(float), st);
  cudaError_t e = launch_pair_table(pt, t->d64, t->Lmax, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    afree(pt, st);
    throw CudaFail{e};
  }
  t->pair32 = pt;
  t->bytes += (size_t)pair_table_entries(t->Lmax) * sizeof(float);
}

void delta_release(DeltaTab* t) {
  if (!t) return;
  std::lock_guard<std::mutex> lk(g_mu);
  if (--t->refs == 0) {
    cudaStream_t st = setup_stream();
    afree(t->raw64, st);
    afree(t->raw32, st);
    afree(t->pair32, st);
    g_tabs.erase(std::remove(g_tabs.begin(), g_tabs.end(), t), g_tabs.end());
    delete t;
  }
}

// launch-list keys of the FP32 contraction tasks: N | (CTA shape << 8)
constexpr int kShapeShift = 8;

// Device-resident launch lists for a set of jobs (one plan = one job).
struct Lists {
  void* mem = nullptr;
  void* desc_w = nullptr;     // ContractDesc<T>[njobs]
  void* desc_phi = nullptr;   // ContractDesc<T>[njobs]
  // (N, or N | shape << kShapeShift for the FP32 contraction, (tiles, count))
  std::vector<std::pair<int, std::pair<void*, int>>> tiles_w;
  void* tiles_phi = nullptr;
  int ntiles_phi = 0;
  static constexpr int NK = 16;  // chirp-z 0..3, direct alpha 4..5, single-FFT beta 6..7, segmented alpha 8..9,
                                 // MW-grid synthesis beta 10..12, half-length beta 13..15
  void* segs[NK] = {};
  int nseg[NK] = {};
  int items[NK] = {};
  int ulogM[NK] = {};  // the segments' common transform length log2 (0: lengths differ)
  // half-length beta kinds (13..15): the segments ordered by transform length,
  // one launch per length {first segment, segments, items, log2 length}, so
  // that each launch runs the kernel compiled for its length
  std::vector<std::array<int, 4>> dct_parts[3];
  int maxlogM = 0;
  int Lmax = 0;
  int odd = 0;  // CZT_ODD_ROWS when a plan of the list samples the MW grid
  int njobs = 0, nbmax = 0, Lrmax = 0;  // f packing of the FP32 contraction (jobs, 32-blocks, rows)
  ~Lists() {
    if (mem) {
      try {
        afree(mem, setup_stream());
      } catch (...) {
      }
    }
  }
};

}  // namespace

struct s2dw_plan_s {
  int L = 0, N = 0, J0 = 0, J = 0, nscale = 0;
  unsigned flags = 0;
  double lam = 0;
  bool fp64 = false;
  int E = 4, TMP = 32;
  std::vector<int> lo, hi, Lj;
  int lend_w = -1, L0 = 0, lphi = 0, Lphi = 1;
  int logM = 0, M = 0;
  int device = 0;
  DeltaTab* tab = nullptr;
  std::vector<double> psi_host, phi_host;
  bool sht = false;                 // companion plan of the spherical harmonic transforms
  s2dw_plan_s* sht_child = nullptr; // created on the first s2dw_sht_* call
  cudaStream_t pst = nullptr;       // private non-blocking stream (set-up, frees)
  cudaEvent_t last_use = nullptr;   // recorded after every call using the plan
  void* ws = nullptr;
  size_t ws_bytes = 0;
  // workspace views
  void* RS = nullptr;
  void* RSphi = nullptr;
  std::vector<void*> Y, X;  // [nscale + 1], last = scaling part
  std::vector<int> Ycols;   // band-limit of each buffer (Lj, last = Lphi)
  void* P = nullptr;
  void* Pphi = nullptr;
  int nbr = 0, nbr_phi = 0, Lp = 0, Lp32 = 0, Lphip = 0, Lphip32 = 0;
  // Tables of one sampling grid (band-limit Lg: 2Lg beta, 2Lg-1 alpha samples).
  struct GridTables {
    int L = 0, logM = 0, M = 0;
    int nb = 0;              // beta samples: 2L (DH), or L (MW grid)
    void* tw = nullptr;
    void* chirp_a = nullptr;
    void* pre_b = nullptr;
    void* post_b = nullptr;
    void* preS_b = nullptr;
    void* postS_b = nullptr;
    void* root_a = nullptr;  // e^{2 pi i t/(2Lg-1)}
    void* pre_mw = nullptr;  // MW beta chirp e^{i pi (m'^2 + m')/(2Lg-1)}, |m'| < Lg
    void* bfft = nullptr;    // e^{i pi m'/(4Lg)} (|m'| < Lg), then q_b (b < 2Lg): single-FFT beta
    void* tw2 = nullptr;     // FFT twiddles of length 2Lg (half-length beta)
    void* Hs = nullptr;      // 4 x M spectra
  };
  bool multires = false;       // every scale on the grid of its own band-limit
  bool mw = false;             // L beta samples per grid (McEwen-Wiaux), not 2L
  std::vector<GridTables> gt;  // one set per distinct grid band-limit
  std::vector<int> grid_of;    // [nscale + 1]: set of scale j (last: scaling part)
  std::vector<int64_t> woff;   // [nscale + 1]: element offset of scale j in W (last: total)
  // segmented chirp-z of scale j (S == 0: one convolution of the grid's length M)
  struct SegTables {
    int logM = 0, P = 0, S = 0;
    void* tw = nullptr;  // twiddles of length 2^logM
    void* Ha = nullptr;  // S analysis spectra of length 2^logM
    void* Hs = nullptr;  // S synthesis spectra
  };
  std::vector<SegTables> seg;  // [nscale + 1]
  // launch methods (s2dw_plan_choices / s2dw_plan_tune): beta_mode[dir] 0 = one
  // FFT of length 4L, 1 = half-length transforms on the grids where they are
  // faster (power-of-two L >= 128; synthesis up to 1024);
  // alpha_mode[dir][j] 0 = direct sums (L_j <= 32), 1 = chirp-z of the grid's
  // length, 2 = segmented chirp-z (where its tables exist); dir 0 = analysis
  int beta_mode[2] = {1, 1};
  std::vector<int> alpha_mode[2];
  // [nscale + 1]: tensor-core basis images of the direct alpha sums (FP32 plans)
  std::vector<void*> tc_ana, tc_syn;
  // FP32 plans: R rows and packed f of the tile-pair contraction
  void* RSp = nullptr;
  void* RSphi_p = nullptr;
  void* fP = nullptr;
  int Lr = 0, Lrphi = 0, Lrf = 0;
  // host copies of the static descriptors (device copies live in `own`)
  std::vector<unsigned char> desc_w_host, desc_phi_host;
  std::vector<TileTask> tiles_w_host, tiles_phi_host;  // FP64 plans
  std::vector<PairTask> ptasks_w_host, ptasks_phi_host;  // FP32 plans
  int pair_shape = kPairShapePair;  // FP32: the contraction's CTA shape (a launch method; N > 5: one tile)
  Lists own;
  // stage timing (s2dw_profile): one set of events per call, up to kProfCalls
  static constexpr int kProfCalls = 256;
  bool prof = false;
  static constexpr int kEvAna = 7, kEvSyn = 8;  // events per call (stages + 1)
  std::vector<cudaEvent_t> ev_ana, ev_syn;      // kProfCalls x kEvAna, kProfCalls x kEvSyn
  int nana = 0, nsyn = 0;
  ~s2dw_plan_s() {
    for (auto e : ev_ana)
      if (e) cudaEventDestroy(e);
    for (auto e : ev_syn)
      if (e) cudaEventDestroy(e);
    delete sht_child;
    if (last_use) {
      cudaEventSynchronize(last_use);  // only this plan's work, not the device
      cudaEventDestroy(last_use);
    }
    if (ws) cudaFreeAsync(ws, pst);
    own.mem = nullptr;
    if (own_mem) cudaFreeAsync(own_mem, pst);
    if (pst) cudaStreamDestroy(pst);  // releases after the queued frees
    delta_release(tab);
  }
  void* own_mem = nullptr;
};

namespace {

// Launch lists of the plan sets seen by the batched entry points.  At most
// kBatchCacheMax entries: beyond that the least recently used one is freed
// once its last launch has completed, unless it was used while its stream was
// being captured into a CUDA graph (the graph keeps reading it, so it lives
// until one of its plans is destroyed).
struct BatchEnt {
  Lists* ls = nullptr;
  uint64_t tick = 0;
  cudaEvent_t done = nullptr;  // recorded after the entry's latest launches
  bool pinned = false;
};
constexpr size_t kBatchCacheMax = 64;
std::mutex g_batch_mu;
std::map<std::vector<s2dw_plan_t>, BatchEnt> g_batch_cache;
uint64_t g_batch_tick = 0;

void free_batch_ent(BatchEnt& e) {
  if (e.done) {
    cudaEventSynchronize(e.done);  // only this entry's launches
    cudaEventDestroy(e.done);
  }
  delete e.ls;
}

void drop_batches_with(s2dw_plan_t p) {
  std::lock_guard<std::mutex> lk(g_batch_mu);
  for (auto it = g_batch_cache.begin(); it != g_batch_cache.end();) {
    if (std::find(it->first.begin(), it->first.end(), p) != it->first.end()) {
      free_batch_ent(it->second);
      it = g_batch_cache.erase(it);
    } else {
      ++it;
    }
  }
}

void evict_batches() {  // g_batch_mu held; called before an insertion
  while (g_batch_cache.size() >= kBatchCacheMax) {  // room for one more
    auto victim = g_batch_cache.end();
    for (auto it = g_batch_cache.begin(); it != g_batch_cache.end(); ++it)
      if (!it->second.pinned && (victim == g_batch_cache.end() || it->second.tick < victim->second.tick))
        victim = it;
    if (victim == g_batch_cache.end()) return;
    free_batch_ent(victim->second);
    g_batch_cache.erase(victim);
  }
}

template <typename T>
void fill_desc(s2dw_plan_s* p, ContractDesc<T>& dw, ContractDesc<T>& dp, const T* delta) {
  std::memset(&dw, 0, sizeof(dw));
  std::memset(&dp, 0, sizeof(dp));
  dw.delta = delta;
  dw.dpair = p->tab->pair32;
  dw.RSp = reinterpret_cast<const float*>(p->RSp);
  dw.fP = reinterpret_cast<const cx<T>*>(p->fP);
  dw.Lr = p->Lr;
  dw.Lrf = p->Lrf;
  dw.RS = reinterpret_cast<const T*>(p->RS);
  dw.P = reinterpret_cast<cx<T>*>(p->P);
  dw.L = p->L;
  dw.Lp = p->Lp;
  dw.Lp32 = p->Lp32;
  dw.nbr = p->nbr;
  dw.N = p->N;
  dw.nslot = 2;
  dw.eta_odd = (p->N % 2 == 0) ? 1 : 0;
  for (int j = 0; j < p->nscale; ++j) {
    dw.Lj[j] = p->Lj[j];
    dw.Y[j] = reinterpret_cast<cx<T>*>(p->Y[j]);
  }
  // l-segments with constant slot occupancy, covering [0, L-1]
  int ns = 0;
  int prev0 = -2, prev1 = -2;
  for (int l = 0; l < p->L; ++l) {
    int s0 = -1, s1 = -1;
    for (int j = 0; j < p->nscale; ++j) {
      if (p->Lj[j] == 0 || l < p->lo[j] || l > p->hi[j]) continue;
      if (j % 2 == 0) s0 = j;
      else s1 = j;
    }
    if (s0 != prev0 || s1 != prev1) {
      dw.seg[ns].lo = l;
      dw.seg[ns].hi = l;
      dw.seg[ns].j[0] = s0;
      dw.seg[ns].j[1] = s1;
      ++ns;
      prev0 = s0;
      prev1 = s1;
    } else {
      dw.seg[ns - 1].hi = l;
    }
  }
  dw.nseg = ns;
  // scaling part: one N = 1 "scale" with kernel Phi on [0, lphi]
  dp.delta = delta;
  dp.dpair = p->tab->pair32;
  dp.RSp = reinterpret_cast<const float*>(p->RSphi_p);
  dp.fP = reinterpret_cast<const cx<T>*>(p->fP);
  dp.Lr = p->Lrphi;
  dp.Lrf = p->Lrf;
  dp.RS = reinterpret_cast<const T*>(p->RSphi);
  dp.P = reinterpret_cast<cx<T>*>(p->Pphi);
  dp.L = p->Lphi;
  dp.Lp = p->Lphip;
  dp.Lp32 = p->Lphip32;
  dp.nbr = p->nbr_phi;
  dp.N = 1;
  dp.nslot = 1;
  dp.eta_odd = 0;
  dp.Lj[0] = p->Lphi;
  dp.Y[0] = reinterpret_cast<cx<T>*>(p->Y[p->nscale]);
  dp.seg[0].lo = 0;
  dp.seg[0].hi = p->Lphi - 1;
  dp.seg[0].j[0] = 0;
  dp.seg[0].j[1] = -1;
  dp.nseg = 1;
}

void build_tiles(int Lband, int lend, int TMP, int prob, std::vector<TileTask>& out) {
  if (Lband <= 0 || lend < 0) return;
  const int nbp = (Lband + TMP - 1) / TMP, nbm = (Lband + TILE - 1) / TILE;
  for (int bp = 0; bp < nbp; ++bp)
    for (int bm = 0; bm < nbm; ++bm) {
      const int ls = std::max(bp * TMP, bm * TILE);
      if (ls > lend) continue;
      out.push_back(TileTask{prob, bp, bm, ls, lend});
    }
}

// Tile pairs (p <= q) of a band Lband with l in [32 q, lend]; a pair whose
// tiles run on separate CTAs (N > 5) becomes two tasks.  Sorted by decreasing
// work (two tiles count double) so that the long ones start first.
// two: one task per pair of tiles (both computed by one CTA, N <= 5), else
// one task per tile
void build_pair_tasks(int Lband, int lend, bool two, int table_Lmax, std::vector<PairTask>& out) {
  out.clear();
  if (Lband <= 0 || lend < 0) return;
  const int nb = (Lband + 31) / 32;
  for (int q = 0; q < nb; ++q)
    for (int p = 0; p <= q; ++p) {
      const int ls = 32 * q;
      if (ls > lend) continue;
      const long long base = pair_run_base(p, q, table_Lmax);
      if (two || p == q) {
        out.push_back(PairTask{0, p, q, ls, lend, 0, base});
      } else {
        out.push_back(PairTask{0, p, q, ls, lend, 0, base});
        out.push_back(PairTask{0, p, q, ls, lend, 1, base});
      }
    }
  auto work = [two](const PairTask& t) { return (long long)(t.lend - t.lstart + 1) * (two && t.p != t.q ? 2 : 1); };
  std::stable_sort(out.begin(), out.end(), [&](const PairTask& a, const PairTask& b) { return work(a) > work(b); });
}

void sort_tiles(std::vector<TileTask>& t) {
  std::stable_sort(t.begin(), t.end(), [](const TileTask& a, const TileTask& b) {
    return (a.lend - a.lstart) > (b.lend - b.lstart);
  });
}

template <typename T>
void build_segs(s2dw_plan_s* p, int job, int kind, std::vector<CztSeg<T>>& out, int& start) {
  // kinds 4 / 5 collect the alpha segments of scales with Lj <= kDirectMaxLjAna
  // (analysis) or kDirectMaxLj (synthesis),
  // kinds 6 / 7 the beta segments of plans whose FFT length M is 4L
  // kinds 8 / 9 the alpha segments of scales with a segmented chirp-z;
  // kinds 10..12 (MW grid only) the synthesis-side resampling of V from the L
  // MW beta samples to the DH beta grid (torus coefficients, then their
  // evaluation on the DH grid by the analysis beta kernels)
  if ((kind == CZT_BETA_MW_DFT || kind == CZT_BETA_RS_FFT || kind == CZT_BETA_RS || kind == CZT_BETA_RS_DCT) &&
      !p->mw)
    return;
  const int base_kind = (kind == CZT_ALPHA_ANA_DIRECT || kind == CZT_ALPHA_ANA_SEG) ? CZT_ALPHA_ANA
                        : (kind == CZT_ALPHA_SYN_DIRECT || kind == CZT_ALPHA_SYN_SEG) ? CZT_ALPHA_SYN
                        : (kind == CZT_BETA_ANA_FFT || kind == CZT_BETA_RS_FFT || kind == CZT_BETA_RS ||
                           kind == CZT_BETA_MW_DFT || kind == CZT_BETA_ANA_DCT || kind == CZT_BETA_RS_DCT)
                            ? CZT_BETA_ANA
                        : (kind == CZT_BETA_SYN_FFT || kind == CZT_BETA_SYN_DCT) ? CZT_BETA_SYN
                                                                                  : kind;
  const bool rs_list = kind == CZT_BETA_RS_FFT || kind == CZT_BETA_RS || kind == CZT_BETA_RS_DCT;
  const bool dct_list = kind == CZT_BETA_ANA_DCT || kind == CZT_BETA_SYN_DCT || kind == CZT_BETA_RS_DCT;
  const bool direct_list = kind == CZT_ALPHA_ANA_DIRECT || kind == CZT_ALPHA_SYN_DIRECT;
  const bool seg_list = kind == CZT_ALPHA_ANA_SEG || kind == CZT_ALPHA_SYN_SEG;
  const bool fft_list = kind == CZT_BETA_ANA_FFT || kind == CZT_BETA_SYN_FFT || kind == CZT_BETA_RS_FFT;
  for (int j = 0; j <= p->nscale; ++j) {
    const bool phi = (j == p->nscale);
    const int Nj = phi ? 1 : p->N;
    const int Lj = p->Ycols[j];
    const s2dw_plan_s::GridTables& G = p->gt[p->grid_of[j]];
    const int L = G.L, n = 2 * L - 1;  // this scale's sampling grid
    // the analysis beta step of an MW plan evaluates at the MW samples (chirp-z only);
    // the DH-grid beta kernels (FFT for power-of-two L) serve DH plans and the MW resampling
    const bool mw_ana_beta = p->mw && base_kind == CZT_BETA_ANA && !rs_list && kind != CZT_BETA_MW_DFT;
    // power-of-two L: half-length transforms (L >= 16) or one FFT of length 4L (L = 8); else chirp-z
    const bool beta_pow2 = (4 * L == G.M) && !mw_ana_beta;
    const int bdir = base_kind == CZT_BETA_SYN ? 1 : 0;
    // mode 1: the half-length transforms on the grids where they measured
    // faster than the length-4L FFT (GB300, N = 3): L >= 128 in the analysis,
    // 128 <= L <= 1024 in the synthesis
    const bool dct_faster = bdir == 0 ? L >= 128 : (L >= 128 && L <= 1024);
    const bool beta_dct = beta_pow2 && L >= 16 && p->beta_mode[bdir] == 1 && dct_faster;
    const bool beta_fft = beta_pow2 && !beta_dct;
    if ((base_kind == CZT_BETA_ANA || base_kind == CZT_BETA_SYN) && kind != CZT_BETA_MW_DFT &&
        (beta_fft != fft_list || beta_dct != dct_list))
      continue;
    const cx<T>* Hs = reinterpret_cast<const cx<T>*>(G.Hs);
    CztSeg<T> s;
    std::memset(&s, 0, sizeof(s));
    s.job = job;
    s.L = L;
    s.Lj = Lj;
    s.N = Nj;
    s.logM = G.logM;
    s.woff = phi ? 0 : p->woff[j];
    s.is_phi = phi ? 1 : 0;
    s.tw = reinterpret_cast<const cx<T>*>(G.tw);
    s.scale = (T)(2.0 * 3.14159265358979323846 / n);
    s.nb = G.nb;
    const bool is_alpha = base_kind == CZT_ALPHA_ANA || base_kind == CZT_ALPHA_SYN;
    const int amode = is_alpha ? p->alpha_mode[base_kind == CZT_ALPHA_SYN ? 1 : 0][j] : -1;
    const bool direct = is_alpha && amode == 0;
    if (direct != direct_list) continue;
    if (is_alpha && !direct && (amode == 2) != seg_list) continue;
    switch (base_kind) {
      case CZT_BETA_ANA:
        s.P = beta_czt_cols(G.logM, sizeof(T) == 8);  // columns per CTA of the chirp-z beta kernels
        s.items = Nj * ((Lj + s.P - 1) / s.P);
        s.buf_in = reinterpret_cast<cx<T>*>(p->Y[j]);
        s.buf_out = reinterpret_cast<cx<T>*>(p->X[j]);
        s.H = Hs + 0 * (size_t)G.M;
        s.pre = reinterpret_cast<const cx<T>*>(G.pre_b);
        s.post = reinterpret_cast<const cx<T>*>(G.post_b);
        if (kind == CZT_BETA_MW_DFT) {  // V [g][b < L][m] -> torus coefficients [g][m][p]
          s.buf_in = reinterpret_cast<cx<T>*>(p->X[j]);
          s.buf_out = reinterpret_cast<cx<T>*>(p->Y[j]);
          s.H = Hs + 2 * (size_t)G.M;   // the alpha synthesis kernel e^{+i pi u^2/n}
          s.pre = reinterpret_cast<const cx<T>*>(G.chirp_a);
          s.post = reinterpret_cast<const cx<T>*>(G.pre_mw);
        } else if (rs_list) {           // coefficients -> the 2L DH samples
          s.nb = 2 * L;
        } else if (p->mw) {             // analysis: the L MW samples beta_b = (2b+1) pi / n
          s.H = Hs + 1 * (size_t)G.M;   // the alpha analysis kernel e^{-i pi u^2/n}
          s.pre = reinterpret_cast<const cx<T>*>(G.pre_mw);
          s.post = reinterpret_cast<const cx<T>*>(G.chirp_a);
        }
        break;
      case CZT_ALPHA_ANA:
        s.items = ((Nj * G.nb + 1) / 2 + alpha_czt_nt(sizeof(T) == 8) - 1) / alpha_czt_nt(sizeof(T) == 8);
        s.buf_in = reinterpret_cast<cx<T>*>(p->X[j]);
        s.H = Hs + 1 * (size_t)G.M;
        s.pre = reinterpret_cast<const cx<T>*>(G.chirp_a);
        s.post = reinterpret_cast<const cx<T>*>(G.chirp_a);
        break;
      case CZT_ALPHA_SYN:
        s.items = ((Nj * G.nb + 1) / 2 + alpha_czt_nt(sizeof(T) == 8) - 1) / alpha_czt_nt(sizeof(T) == 8);
        s.buf_out = reinterpret_cast<cx<T>*>(p->X[j]);
        s.H = Hs + 2 * (size_t)G.M;
        s.pre = reinterpret_cast<const cx<T>*>(G.chirp_a);
        s.post = reinterpret_cast<const cx<T>*>(G.chirp_a);
        break;
      case CZT_BETA_SYN:
        s.P = beta_czt_cols(G.logM, sizeof(T) == 8);  // columns per CTA of the chirp-z beta kernels
        s.items = Nj * ((Lj + s.P - 1) / s.P);
        s.nb = 2 * L;  // DH quadrature (an MW plan resamples V to the DH grid first)
        s.buf_in = reinterpret_cast<cx<T>*>(p->X[j]);
        s.buf_out = reinterpret_cast<cx<T>*>(p->Y[j]);
        s.H = Hs + 3 * (size_t)G.M;
        s.pre = reinterpret_cast<const cx<T>*>(G.preS_b);
        s.post = reinterpret_cast<const cx<T>*>(G.postS_b);
        break;
    }
    if (fft_list) {
      const int ntb = beta_fft_nt(sizeof(T) == 8);
      s.items = Nj * ((Lj + ntb - 1) / ntb);
      s.pre = reinterpret_cast<const cx<T>*>(G.bfft);
      s.post = reinterpret_cast<const cx<T>*>(G.bfft) + (2 * L - 1);
    }
    if (dct_list) {
      const int cols = 4096 / (2 * L);  // transforms of length 2L per CTA
      s.items = Nj * ((Lj + cols - 1) / cols);
      s.tw = reinterpret_cast<const cx<T>*>(G.tw2);
      s.pre = reinterpret_cast<const cx<T>*>(G.bfft);
      s.post = reinterpret_cast<const cx<T>*>(G.bfft) + (2 * L - 1);
    }
    if (seg_list) {
      const auto& sgt = p->seg[j];
      const int groups = 1 << (12 - sgt.logM);  // row pairs per CTA (one per group of M'/16 threads)
      s.items = ((Nj * G.nb + 1) / 2 + groups - 1) / groups;
      s.logM = sgt.logM;
      s.tw = reinterpret_cast<const cx<T>*>(sgt.tw);
      s.H = reinterpret_cast<const cx<T>*>(base_kind == CZT_ALPHA_ANA ? sgt.Ha : sgt.Hs);
      s.P = sgt.P;
      s.nsegs = sgt.S;
    }
    if (direct) {
      const bool syn = base_kind == CZT_ALPHA_SYN;
      if (sizeof(T) == sizeof(float)) {  // tensor cores: the plan's basis image of this scale
        s.items = alpha_tc_items(L, Nj * G.nb, syn);
        s.H = reinterpret_cast<const cx<T>*>(syn ? p->tc_syn[j] : p->tc_ana[j]);
      } else if (!syn) {
        s.items = ((n + kAgCols - 1) / kAgCols) * ((Nj * G.nb + kAgChunk - 1) / kAgChunk);
      } else {
        s.items = (Nj * G.nb + direct_rows_syn(sizeof(T) == 8) - 1) / direct_rows_syn(sizeof(T) == 8);
      }
      s.pre = reinterpret_cast<const cx<T>*>(G.root_a);
    }
    if (s.items <= 0) continue;
    s.start = start;
    start += s.items;
    out.push_back(s);
  }
}

// Build the device launch lists for a set of plans (same precision).
template <typename T>
Lists* build_lists(const std::vector<s2dw_plan_t>& plans) {
  // FP32 plans run the tile-pair contraction (PairTask), FP64 plans the
  // eighth-domain one (TileTask)
  using Task = typename std::conditional<sizeof(T) == sizeof(float), PairTask, TileTask>::type;
  const int nj = (int)plans.size();
  std::vector<ContractDesc<T>> dw(nj), dp(nj);
  std::map<int, std::vector<Task>> tw_byN;
  std::vector<Task> tphi;
  std::vector<CztSeg<T>> segs[Lists::NK];
  int start[Lists::NK] = {};
  Lists* ls = new Lists();
  ls->njobs = nj;
  for (int i = 0; i < nj; ++i) {
    s2dw_plan_s* p = plans[i];
    std::memcpy(&dw[i], p->desc_w_host.data(), sizeof(ContractDesc<T>));
    std::memcpy(&dp[i], p->desc_phi_host.data(), sizeof(ContractDesc<T>));
    const std::vector<Task>* tws;
    const std::vector<Task>* tps;
    if constexpr (sizeof(T) == sizeof(float)) {
      tws = &p->ptasks_w_host;
      tps = &p->ptasks_phi_host;
    } else {
      tws = &p->tiles_w_host;
      tps = &p->tiles_phi_host;
    }
    const int key = p->N | ((sizeof(T) == sizeof(float)) ? (p->pair_shape << kShapeShift) : 0);
    for (Task t : *tws) {
      t.prob = i;
      tw_byN[key].push_back(t);
    }
    for (Task t : *tps) {
      t.prob = i;
      tphi.push_back(t);
    }
    for (int k = 0; k < Lists::NK; ++k) build_segs<T>(p, i, k, segs[k], start[k]);
    ls->maxlogM = std::max(ls->maxlogM, p->logM);
    ls->Lmax = std::max(ls->Lmax, p->L);
    ls->nbmax = std::max(ls->nbmax, (p->L + 31) / 32);
    ls->Lrmax = std::max(ls->Lrmax, p->Lrf);
    if (p->mw) ls->odd = CZT_ODD_ROWS;
  }
  for (int k = CZT_BETA_ANA_DCT; k <= CZT_BETA_RS_DCT; ++k) {
    std::stable_sort(segs[k].begin(), segs[k].end(),
                     [](const CztSeg<T>& a, const CztSeg<T>& b) { return a.logM < b.logM; });
    auto& parts = ls->dct_parts[k - CZT_BETA_ANA_DCT];
    int first = 0, st = 0;
    for (int i = 0; i <= (int)segs[k].size(); ++i) {
      if (i == (int)segs[k].size() || (i > first && segs[k][i].logM != segs[k][first].logM)) {
        if (i > first) parts.push_back({first, i - first, st, segs[k][first].logM});
        if (i == (int)segs[k].size()) break;
        first = i;
        st = 0;
      }
      segs[k][i].start = st;  // CTA indices restart in every part
      st += segs[k][i].items;
    }
  }
  for (int k = 0; k < Lists::NK; ++k) {
    int u = segs[k].empty() ? 0 : segs[k][0].logM;
    for (const CztSeg<T>& sg : segs[k])
      if (sg.logM != u) u = 0;
    ls->ulogM[k] = u;
  }
  // longest tasks first (a CTA computing both tiles of a pair counts double)
  auto by_work = [](std::vector<Task>& v, int key) {
    if constexpr (sizeof(T) == sizeof(float)) {
      const bool two = (key >> kShapeShift) == kPairShapePair;
      auto work = [two](const PairTask& t) {
        return (long long)(t.lend - t.lstart + 1) * (two && t.p != t.q ? 2 : 1);
      };
      std::stable_sort(v.begin(), v.end(), [&](const PairTask& a, const PairTask& b) { return work(a) > work(b); });
    } else {
      (void)key;
      sort_tiles(v);
    }
  };
  for (auto& kv : tw_byN) by_work(kv.second, kv.first);
  by_work(tphi, 1);
  // one allocation for everything
  size_t off = 0;
  const size_t o_dw = off;
  off = align256(off + nj * sizeof(ContractDesc<T>));
  const size_t o_dp = off;
  off = align256(off + nj * sizeof(ContractDesc<T>));
  std::vector<size_t> o_tw;
  for (auto& kv : tw_byN) {
    o_tw.push_back(off);
    off = align256(off + kv.second.size() * sizeof(Task));
  }
  const size_t o_tp = off;
  off = align256(off + tphi.size() * sizeof(Task));
  size_t o_sg[Lists::NK];
  for (int k = 0; k < Lists::NK; ++k) {
    o_sg[k] = off;
    off = align256(off + segs[k].size() * sizeof(CztSeg<T>));
  }
  std::vector<unsigned char> host(off, 0);
  std::memcpy(host.data() + o_dw, dw.data(), nj * sizeof(ContractDesc<T>));
  std::memcpy(host.data() + o_dp, dp.data(), nj * sizeof(ContractDesc<T>));
  int q = 0;
  for (auto& kv : tw_byN) {
    std::memcpy(host.data() + o_tw[q], kv.second.data(), kv.second.size() * sizeof(Task));
    ++q;
  }
  if (!tphi.empty()) std::memcpy(host.data() + o_tp, tphi.data(), tphi.size() * sizeof(Task));
  for (int k = 0; k < Lists::NK; ++k)
    if (!segs[k].empty()) std::memcpy(host.data() + o_sg[k], segs[k].data(), segs[k].size() * sizeof(CztSeg<T>));
  try {
    cudaStream_t st = setup_stream();
    amalloc(&ls->mem, off, st);
    ck(cudaMemcpyAsync(ls->mem, host.data(), off, cudaMemcpyHostToDevice, st));
    ck(cudaStreamSynchronize(st));  // host staging buffer is local
  } catch (...) {
    delete ls;
    throw;
  }
  char* base = reinterpret_cast<char*>(ls->mem);
  ls->desc_w = base + o_dw;
  ls->desc_phi = base + o_dp;
  q = 0;
  for (auto& kv : tw_byN) {
    ls->tiles_w.push_back({kv.first, {base + o_tw[q], (int)kv.second.size()}});
    ++q;
  }
  ls->tiles_phi = base + o_tp;
  ls->ntiles_phi = (int)tphi.size();
  for (int k = 0; k < Lists::NK; ++k) {
    ls->segs[k] = base + o_sg[k];
    ls->nseg[k] = (int)segs[k].size();
    ls->items[k] = start[k];
  }
  return ls;
}

inline void rec(cudaEvent_t* ev, int i, cudaStream_t st) {
  if (ev) cudaEventRecord(ev[i], st);
}

// True while `st` is being captured into a CUDA graph.  The library's own
// events (last use, stage timing) are not recorded then: a captured record
// would tie the plan's events to the caller's graph (and cannot be waited
// on), so keeping a plan alive while a graph that captured it may still run
// is the caller's responsibility, as for the buffers it passed.
inline bool capturing(cudaStream_t st) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}
inline void mark_use(s2dw_plan_t p, cudaStream_t st) {
  if (!capturing(st)) cudaEventRecord(p->last_use, st);
}

// Analysis stages: [contraction + gamma | scaling contraction | beta | alpha chirp-z full-band | segmented
// | alpha direct].
// the half-length beta launches of a kind, one per transform length
template <typename T>
void launch_dct_parts(const Lists& ls, int kind, const CallPtrs& ptrs, cudaStream_t st) {
  const CztSeg<T>* segs = reinterpret_cast<const CztSeg<T>*>(ls.segs[kind]);
  for (const auto& pt : ls.dct_parts[kind - CZT_BETA_ANA_DCT])
    launch_czt<T>(kind, segs + pt[0], pt[1], pt[2], ls.maxlogM, ptrs, st, pt[3]);
}

template <typename T>
void run_analysis(const Lists& ls, const CallPtrs& ptrs, cudaStream_t st, cudaEvent_t* ev = nullptr) {
  const ContractDesc<T>* dw = reinterpret_cast<const ContractDesc<T>*>(ls.desc_w);
  const ContractDesc<T>* dp = reinterpret_cast<const ContractDesc<T>*>(ls.desc_phi);
  rec(ev, 0, st);
  if constexpr (sizeof(T) == sizeof(float)) {
    launch_fpack(dw, ls.njobs, ls.nbmax, ls.Lrmax, ptrs, st);
    for (auto& t : ls.tiles_w)
      launch_contract_pair(t.first & 0xff, 2, false, t.first >> kShapeShift, dw,
                           reinterpret_cast<const PairTask*>(t.second.first), t.second.second, ptrs, st);
    rec(ev, 1, st);
    launch_contract_pair(1, 1, false, kPairShapePair, dp, reinterpret_cast<const PairTask*>(ls.tiles_phi), ls.ntiles_phi, ptrs,
                         st);
  } else {
    for (auto& t : ls.tiles_w)
      launch_contract<T>(t.first, 2, false, dw, reinterpret_cast<const TileTask*>(t.second.first), t.second.second,
                         ptrs, st);
    rec(ev, 1, st);
    launch_contract<T>(1, 1, false, dp, reinterpret_cast<const TileTask*>(ls.tiles_phi), ls.ntiles_phi, ptrs, st);
  }
  rec(ev, 2, st);
  launch_czt<T>(CZT_BETA_ANA, reinterpret_cast<const CztSeg<T>*>(ls.segs[0]), ls.nseg[0], ls.items[0], ls.maxlogM,
                ptrs, st, ls.ulogM[0]);
  launch_czt<T>(CZT_BETA_ANA_FFT, reinterpret_cast<const CztSeg<T>*>(ls.segs[6]), ls.nseg[6], ls.items[6],
                ls.maxlogM, ptrs, st, ls.ulogM[6]);
  launch_dct_parts<T>(ls, CZT_BETA_ANA_DCT, ptrs, st);
  rec(ev, 3, st);
  launch_czt<T>(CZT_ALPHA_ANA | ls.odd, reinterpret_cast<const CztSeg<T>*>(ls.segs[1]), ls.nseg[1], ls.items[1],
                ls.maxlogM, ptrs, st, ls.ulogM[1]);
  rec(ev, 4, st);
  launch_czt<T>(CZT_ALPHA_ANA_SEG | ls.odd, reinterpret_cast<const CztSeg<T>*>(ls.segs[8]), ls.nseg[8], ls.items[8],
                ls.maxlogM, ptrs, st, ls.ulogM[8]);
  rec(ev, 5, st);
  launch_czt<T>(CZT_ALPHA_ANA_DIRECT, reinterpret_cast<const CztSeg<T>*>(ls.segs[4]), ls.nseg[4], ls.items[4],
                ls.maxlogM, ptrs, st, ls.ulogM[4]);
  rec(ev, 6, st);
}

// Synthesis stages: [alpha direct | alpha chirp-z full-band | segmented | beta | contraction | scaling
// contraction | reduction].
template <typename T>
void run_synthesis(const Lists& ls, const CallPtrs& ptrs, const ReduceJobs& rj, int njobs, cudaStream_t st,
                   cudaEvent_t* ev = nullptr) {
  const ContractDesc<T>* dw = reinterpret_cast<const ContractDesc<T>*>(ls.desc_w);
  const ContractDesc<T>* dp = reinterpret_cast<const ContractDesc<T>*>(ls.desc_phi);
  rec(ev, 0, st);
  launch_czt<T>(CZT_ALPHA_SYN_DIRECT, reinterpret_cast<const CztSeg<T>*>(ls.segs[5]), ls.nseg[5], ls.items[5],
                ls.maxlogM, ptrs, st, ls.ulogM[5]);
  rec(ev, 1, st);
  launch_czt<T>(CZT_ALPHA_SYN, reinterpret_cast<const CztSeg<T>*>(ls.segs[2]), ls.nseg[2], ls.items[2], ls.maxlogM,
                ptrs, st, ls.ulogM[2]);
  rec(ev, 2, st);
  launch_czt<T>(CZT_ALPHA_SYN_SEG | ls.odd, reinterpret_cast<const CztSeg<T>*>(ls.segs[9]), ls.nseg[9], ls.items[9],
                ls.maxlogM, ptrs, st, ls.ulogM[9]);
  rec(ev, 3, st);
  // MW grid: V from its L beta samples to the DH grid (torus coefficients, then the DH samples)
  launch_czt<T>(CZT_BETA_MW_DFT, reinterpret_cast<const CztSeg<T>*>(ls.segs[10]), ls.nseg[10], ls.items[10],
                ls.maxlogM, ptrs, st, ls.ulogM[10]);
  launch_czt<T>(CZT_BETA_RS_FFT, reinterpret_cast<const CztSeg<T>*>(ls.segs[11]), ls.nseg[11], ls.items[11],
                ls.maxlogM, ptrs, st, ls.ulogM[11]);
  launch_dct_parts<T>(ls, CZT_BETA_RS_DCT, ptrs, st);
  launch_czt<T>(CZT_BETA_RS, reinterpret_cast<const CztSeg<T>*>(ls.segs[12]), ls.nseg[12], ls.items[12],
                ls.maxlogM, ptrs, st, ls.ulogM[12]);
  launch_czt<T>(CZT_BETA_SYN, reinterpret_cast<const CztSeg<T>*>(ls.segs[3]), ls.nseg[3], ls.items[3], ls.maxlogM,
                ptrs, st, ls.ulogM[3]);
  launch_czt<T>(CZT_BETA_SYN_FFT, reinterpret_cast<const CztSeg<T>*>(ls.segs[7]), ls.nseg[7], ls.items[7],
                ls.maxlogM, ptrs, st, ls.ulogM[7]);
  launch_dct_parts<T>(ls, CZT_BETA_SYN_DCT, ptrs, st);
  rec(ev, 4, st);
  if constexpr (sizeof(T) == sizeof(float)) {
    for (auto& t : ls.tiles_w)
      launch_contract_pair(t.first & 0xff, 2, true, t.first >> kShapeShift, dw,
                           reinterpret_cast<const PairTask*>(t.second.first), t.second.second, ptrs, st);
    rec(ev, 5, st);
    launch_contract_pair(1, 1, true, kPairShapePair, dp, reinterpret_cast<const PairTask*>(ls.tiles_phi), ls.ntiles_phi, ptrs,
                         st);
  } else {
    for (auto& t : ls.tiles_w)
      launch_contract<T>(t.first, 2, true, dw, reinterpret_cast<const TileTask*>(t.second.first), t.second.second,
                         ptrs, st);
    rec(ev, 5, st);
    launch_contract<T>(1, 1, true, dp, reinterpret_cast<const TileTask*>(ls.tiles_phi), ls.ntiles_phi, ptrs, st);
  }
  rec(ev, 6, st);
  launch_syn_reduce<T>(rj, njobs, ls.Lmax, st);
  rec(ev, 7, st);
}

// (Re)builds the plan's own launch lists from its current methods; the
// previous lists are freed once the plan's private stream is idle.
template <typename T>
void own_lists_build(s2dw_plan_s* p) {
  Lists* ls = build_lists<T>(std::vector<s2dw_plan_t>{p});
  if (p->own_mem) cudaFreeAsync(p->own_mem, p->pst);
  // move into the plan (the plan frees the list memory at destruction)
  p->own_mem = ls->mem;
  p->own.mem = nullptr;
  ls->mem = nullptr;
  p->own.desc_w = ls->desc_w;
  p->own.desc_phi = ls->desc_phi;
  p->own.tiles_w = ls->tiles_w;
  p->own.tiles_phi = ls->tiles_phi;
  p->own.ntiles_phi = ls->ntiles_phi;
  for (int k = 0; k < Lists::NK; ++k) {
    p->own.segs[k] = ls->segs[k];
    p->own.nseg[k] = ls->nseg[k];
    p->own.items[k] = ls->items[k];
    p->own.ulogM[k] = ls->ulogM[k];
  }
  for (int k = 0; k < 3; ++k) p->own.dct_parts[k] = ls->dct_parts[k];
  p->own.maxlogM = ls->maxlogM;
  p->own.Lmax = ls->Lmax;
  p->own.odd = ls->odd;
  p->own.njobs = ls->njobs;
  p->own.nbmax = ls->nbmax;
  p->own.Lrmax = ls->Lrmax;
  delete ls;
}

template <typename T>
void plan_build_typed(s2dw_plan_s* p, const double* kap_d, const double* phi_d, const double* sabs_d,
                      const double* q_d, cudaStream_t st) {
  const int L = p->L, N = p->N;
  // ---- workspace layout ----
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const bool pairc = sizeof(T) == sizeof(float);  // tile-pair contraction (FP32 plans)
  const int NH = (N + 1) / 2;
  p->Lr = L + kPairPadL;  // read-ahead rows of the tile-pair contraction
  p->Lrphi = p->Lphi + kPairPadL;
  p->Lrf = L + kPairPadL;
  const int nbw = (L + 31) / 32, nbp = (p->Lphi + 31) / 32;
  const size_t o_RS = pairc ? take(0) : take((size_t)L * 2 * NH * p->Lp * sizeof(T));
  const size_t o_RSphi = pairc ? take(0) : take((size_t)p->Lphi * p->Lphip * sizeof(T));
  const size_t o_RSp = pairc ? take((size_t)nbw * p->Lr * 2 * NH * 32 * sizeof(float)) : take(0);
  const size_t o_RSphi_p = pairc ? take((size_t)nbp * p->Lrphi * 32 * sizeof(float)) : take(0);
  const size_t o_fP = pairc ? take((size_t)nbw * p->Lrf * 32 * sizeof(cx<T>)) : take(0);
  std::vector<size_t> o_Y(p->nscale + 1), o_X(p->nscale + 1);
  for (int j = 0; j <= p->nscale; ++j) {
    const int Nj = (j == p->nscale) ? 1 : N;
    const int Lj = p->Ycols[j];
    o_Y[j] = take((size_t)Nj * Lj * Lj * sizeof(cx<T>));
    o_X[j] = take((size_t)Nj * 2 * p->gt[p->grid_of[j]].L * Lj * sizeof(cx<T>));
  }
  const size_t o_P = take((size_t)p->nbr * L * p->Lp32 * sizeof(cx<T>));
  const size_t o_Pphi = take((size_t)p->nbr_phi * p->Lphi * p->Lphip32 * sizeof(cx<T>));
  // per grid: twiddles, chirps, roots, beta phases and weights, spectra
  struct GridOff { size_t tw, ca, pb, qb, pS, qS, root, bf, H, pm, tw2; };
  std::vector<GridOff> go(p->gt.size());
  for (size_t g = 0; g < p->gt.size(); ++g) {
    const int Lg = p->gt[g].L, ng = 2 * Lg - 1, Mg = p->gt[g].M;
    go[g].tw = take((size_t)Mg * sizeof(cx<T>));
    go[g].ca = take((size_t)ng * sizeof(cx<T>));
    go[g].pb = take((size_t)(2 * Lg - 1) * sizeof(cx<T>));
    go[g].qb = take((size_t)2 * Lg * sizeof(cx<T>));
    go[g].pS = take((size_t)2 * Lg * sizeof(cx<T>));
    go[g].qS = take((size_t)(2 * Lg - 1) * sizeof(cx<T>));
    go[g].root = take((size_t)ng * sizeof(cx<T>));
    go[g].bf = take((size_t)(4 * Lg - 1) * sizeof(cx<T>));
    go[g].H = take((size_t)4 * Mg * sizeof(cx<T>));
    go[g].pm = take((size_t)ng * sizeof(cx<T>));
    go[g].tw2 = take((size_t)twiddle_entries(p->gt[g].logM - 1) * sizeof(cx<T>));
  }
  // segmented chirp-z tables of the scales that use it (chirp-z bands only)
  p->seg.assign(p->nscale + 1, s2dw_plan_s::SegTables());
  struct SegOff { size_t tw, Ha, Hs; };
  std::vector<SegOff> so(p->nscale + 1);
  for (int j = 0; j <= p->nscale; ++j) {
    const auto& G = p->gt[p->grid_of[j]];
    const int Lj = p->Ycols[j];
    if (Lj <= kDirectMaxLj) continue;  // direct sums
    auto& sgt = p->seg[j];
    seg_choice(G.L, Lj, G.logM, sgt.logM, sgt.P, sgt.S);
    if (sgt.S == 0) continue;
    const size_t Ms = (size_t)1 << sgt.logM;
    so[j].tw = take((size_t)twiddle_entries(sgt.logM) * sizeof(cx<T>));
    so[j].Ha = take((size_t)sgt.S * Ms * sizeof(cx<T>));
    so[j].Hs = take((size_t)sgt.S * Ms * sizeof(cx<T>));
  }
  // default launch methods: direct sums for L_j <= 32, segmented chirp-z where it
  // was chosen above, else the grid's chirp-z
  for (int d = 0; d < 2; ++d) {
    p->alpha_mode[d].assign(p->nscale + 1, 1);
    for (int j = 0; j <= p->nscale; ++j) {
      const int Lj = p->Ycols[j];
      if (Lj <= (d == 0 ? kDirectMaxLjAna : kDirectMaxLj)) p->alpha_mode[d][j] = 0;
      else if (p->seg[j].S > 0) p->alpha_mode[d][j] = 2;
    }
  }
  // tensor-core basis images of the direct alpha sums (FP32 plans)
  std::vector<size_t> o_ta(p->nscale + 1, SIZE_MAX), o_ts(p->nscale + 1, SIZE_MAX);
  if (sizeof(T) == sizeof(float)) {
    for (int j = 0; j <= p->nscale; ++j) {
      const int Lj = p->Ycols[j], Lg = p->gt[p->grid_of[j]].L;
      if (Lj <= 0) continue;
      if (Lj <= kDirectMaxLjAna) o_ta[j] = take(alpha_tc_table_floats(Lg, Lj, false) * sizeof(float));
      if (Lj <= kDirectMaxLj) o_ts[j] = take(alpha_tc_table_floats(Lg, Lj, true) * sizeof(float));
    }
  }
  p->ws_bytes = off;
  amalloc(&p->ws, off, st);
  char* b = reinterpret_cast<char*>(p->ws);
  p->RS = pairc ? nullptr : b + o_RS;
  p->RSphi = pairc ? nullptr : b + o_RSphi;
  p->RSp = pairc ? b + o_RSp : nullptr;
  p->RSphi_p = pairc ? b + o_RSphi_p : nullptr;
  p->fP = pairc ? b + o_fP : nullptr;
  p->Y.resize(p->nscale + 1);
  p->X.resize(p->nscale + 1);
  for (int j = 0; j <= p->nscale; ++j) {
    p->Y[j] = b + o_Y[j];
    p->X[j] = b + o_X[j];
  }
  p->P = b + o_P;
  p->Pphi = b + o_Pphi;
  for (size_t g = 0; g < p->gt.size(); ++g) {
    auto& G = p->gt[g];
    G.tw = b + go[g].tw;
    G.chirp_a = b + go[g].ca;
    G.pre_b = b + go[g].pb;
    G.post_b = b + go[g].qb;
    G.preS_b = b + go[g].pS;
    G.postS_b = b + go[g].qS;
    G.root_a = b + go[g].root;
    G.bfft = b + go[g].bf;
    G.Hs = b + go[g].H;
    G.pre_mw = b + go[g].pm;
    G.tw2 = b + go[g].tw2;
  }
  for (int j = 0; j <= p->nscale; ++j) {
    auto& sgt = p->seg[j];
    if (sgt.S == 0) continue;
    sgt.tw = b + so[j].tw;
    sgt.Ha = b + so[j].Ha;
    sgt.Hs = b + so[j].Hs;
  }
  p->tc_ana.assign(p->nscale + 1, nullptr);
  p->tc_syn.assign(p->nscale + 1, nullptr);
  for (int j = 0; j <= p->nscale; ++j) {
    const int Lj = p->Ycols[j], Lg = p->gt[p->grid_of[j]].L;
    if (o_ta[j] != SIZE_MAX) {
      p->tc_ana[j] = b + o_ta[j];
      ck(alpha_tc_build_table(reinterpret_cast<float*>(p->tc_ana[j]), Lg, Lj, false, st));
    }
    if (o_ts[j] != SIZE_MAX) {
      p->tc_syn[j] = b + o_ts[j];
      ck(alpha_tc_build_table(reinterpret_cast<float*>(p->tc_syn[j]), Lg, Lj, true, st));
    }
  }

  // ---- R tables ----
  std::vector<int> slot_w((size_t)L * 2, -1), slot_p(p->Lphi, 0);
  for (int l = 0; l < L; ++l)
    for (int j = 0; j < p->nscale; ++j)
      if (p->Lj[j] > 0 && l >= p->lo[j] && l <= p->hi[j]) slot_w[(size_t)l * 2 + (j % 2)] = j;
  int* slot_d = nullptr;
  amalloc(&slot_d, (slot_w.size() + slot_p.size()) * sizeof(int), st);
  ck(cudaMemcpyAsync(slot_d, slot_w.data(), slot_w.size() * sizeof(int), cudaMemcpyHostToDevice, st));
  ck(cudaMemcpyAsync(slot_d + slot_w.size(), slot_p.data(), slot_p.size() * sizeof(int), cudaMemcpyHostToDevice,
                     st));
  if (pairc) {
    ck(launch_rtable_pair(reinterpret_cast<float*>(p->RSp), p->tab->d64, kap_d, sabs_d, slot_d, L, p->Lr, N, 2, L,
                          st));
    ck(launch_rtable_pair(reinterpret_cast<float*>(p->RSphi_p), p->tab->d64, phi_d, nullptr, slot_d + slot_w.size(),
                          p->Lphi, p->Lrphi, 1, 1, L, st));
  } else {
    ck(launch_rtable<T>(reinterpret_cast<T*>(p->RS), p->tab->d64, kap_d, sabs_d, slot_d, L, p->Lp, N, 2, L, st));
    ck(launch_rtable<T>(reinterpret_cast<T*>(p->RSphi), p->tab->d64, phi_d, nullptr, slot_d + slot_w.size(),
                        p->Lphi, p->Lphip, 1, 1, L, st));
  }
  // ---- chirp tables of every grid (float64, then the working precision) ----
  double2* t64 = nullptr;
  double* qg = nullptr;
  {
    size_t need = 0;
    for (const auto& G : p->gt) {
      const size_t Lg = G.L, ng = 2 * Lg - 1;
      need = std::max(need, (size_t)G.M + ng + (2 * Lg - 1) + 2 * Lg + 2 * Lg + (2 * Lg - 1) + ng + (4 * Lg - 1) +
                                4 * (size_t)G.M);
    }
    amalloc(&t64, need * sizeof(double2), st);
    amalloc(&qg, (size_t)2 * p->gt.back().L * sizeof(double), st);
  }
  for (auto& G : p->gt) {
    const int Lg = G.L, ng = 2 * Lg - 1, Mg = G.M;
    double2* tw64 = t64;
    double2* ca64 = tw64 + Mg;
    double2* pb64 = ca64 + ng;
    double2* qb64 = pb64 + (2 * Lg - 1);
    double2* pS64 = qb64 + 2 * Lg;
    double2* qS64 = pS64 + 2 * Lg;
    double2* rt64 = qS64 + (2 * Lg - 1);
    double2* bf64 = rt64 + ng;
    double2* H64 = bf64 + (4 * Lg - 1);
    const double* q_g = q_d;  // the plan's own grid reuses its weights
    if (Lg != L) {
      ck(launch_dh_weights(qg, Lg, st));
      q_g = qg;
    }
    ck(launch_chirp_build64(tw64, ca64, pb64, qb64, pS64, qS64, rt64, bf64, H64, q_g, Lg, G.logM, st));
    auto put = [&](void* dst, const double2* src, int64_t cnt) {
      if (sizeof(T) == sizeof(double))
        ck(cudaMemcpyAsync(dst, src, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
      else
        ck(launch_to_prec<float>(reinterpret_cast<float2*>(dst), src, cnt, st));
    };
    put(G.tw, tw64, Mg);
    put(G.chirp_a, ca64, ng);
    put(G.pre_b, pb64, 2 * Lg - 1);
    put(G.post_b, qb64, 2 * Lg);
    put(G.preS_b, pS64, 2 * Lg);
    put(G.postS_b, qS64, 2 * Lg - 1);
    put(G.root_a, rt64, ng);
    put(G.bfft, bf64, 4 * Lg - 1);
    put(G.Hs, H64, (int64_t)4 * Mg);
    ck(launch_mw_pre64(tw64, Lg, st));  // reuse the scratch: the grid's tables are converted above
    put(G.pre_mw, tw64, ng);
    ck(launch_twiddles64(tw64, G.logM - 1, st));  // length 2Lg (half-length beta transforms)
    put(G.tw2, tw64, twiddle_entries(G.logM - 1));
  }
  {
    size_t need = 0;
    for (const auto& sgt : p->seg)
      if (sgt.S)
        need = std::max(need, (size_t)twiddle_entries(sgt.logM) + 2 * (size_t)sgt.S * ((size_t)1 << sgt.logM));
    double2* s64 = nullptr;
    if (need) amalloc(&s64, need * sizeof(double2), st);
    for (int j = 0; j <= p->nscale; ++j) {
      const auto& sgt = p->seg[j];
      if (sgt.S == 0) continue;
      const auto& G = p->gt[p->grid_of[j]];
      const int64_t Ms = (int64_t)1 << sgt.logM, ntw = twiddle_entries(sgt.logM);
      double2* tw64 = s64;
      double2* ha64 = tw64 + ntw;
      double2* hs64 = ha64 + sgt.S * Ms;
      ck(launch_seg_build64(tw64, ha64, hs64, G.L, p->Ycols[j], sgt.logM, sgt.P, sgt.S, st));
      auto put = [&](void* dst, const double2* src, int64_t cnt) {
        if (sizeof(T) == sizeof(double))
          ck(cudaMemcpyAsync(dst, src, (size_t)cnt * sizeof(double2), cudaMemcpyDeviceToDevice, st));
        else
          ck(launch_to_prec<float>(reinterpret_cast<float2*>(dst), src, cnt, st));
      };
      put(sgt.tw, tw64, ntw);
      put(sgt.Ha, ha64, sgt.S * Ms);
      put(sgt.Hs, hs64, sgt.S * Ms);
    }
    afree(s64, st);
  }
  afree(qg, st);
  afree(t64, st);
  afree(slot_d, st);
  ck(cudaStreamSynchronize(st));  // slot_w / slot_p host vectors are local

  // ---- descriptors, tiles, launch lists ----
  if (pairc) {
    delta_pair_ensure(p->tab, st);
    kernels_prepare(false, true);
  }
  ContractDesc<T> dw, dp;
  const T* delta = (sizeof(T) == sizeof(double)) ? reinterpret_cast<const T*>(p->tab->d64)
                                                 : reinterpret_cast<const T*>(p->tab->d32);
  fill_desc<T>(p, dw, dp, delta);
  p->desc_w_host.assign(reinterpret_cast<unsigned char*>(&dw), reinterpret_cast<unsigned char*>(&dw) + sizeof(dw));
  p->desc_phi_host.assign(reinterpret_cast<unsigned char*>(&dp), reinterpret_cast<unsigned char*>(&dp) + sizeof(dp));
  if (pairc) {
    // default CTA shape (measured on GB300): below about 3 pairs per SM one
    // tile per CTA with every value in registers; above it both tiles of a
    // pair (each Delta block read once) for N >= 4, one tile at two CTAs per
    // SM for N <= 3
    {
      int dev = 0, sms = 0;
      ck(cudaGetDevice(&dev));
      ck(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
      const long long nbk = (p->L0 + 31) / 32, npairs = nbk * (nbk + 1) / 2;
      if (!pair_two_tiles(N) || npairs < 3LL * sms) p->pair_shape = kPairShapeTile;
      else p->pair_shape = N >= 4 ? kPairShapePair : kPairShapeTile2;
    }
    build_pair_tasks(p->L0, p->lend_w, p->pair_shape == kPairShapePair, p->tab->Lmax, p->ptasks_w_host);
    build_pair_tasks(p->Lphi, p->lphi, true, p->tab->Lmax, p->ptasks_phi_host);
  } else {
    build_tiles(p->L0, p->lend_w, p->TMP, 0, p->tiles_w_host);
    build_tiles(p->Lphi, p->lphi, p->TMP, 0, p->tiles_phi_host);
    sort_tiles(p->tiles_w_host);
    sort_tiles(p->tiles_phi_host);
  }
  own_lists_build<T>(p);
  // the cap covers every plan size (M <= 8192 for L <= 2048), so plans of
  // different sizes can share a batched launch
  kernels_prepare(sizeof(T) == sizeof(double), false);
}

// sht_mode: the companion plan of s2dw_sht_*: no wavelet scales, N = 1 and
// Phi_l = sqrt((2l+1)/(4 pi)) for every l < L, so that its scaling part is
// the spherical harmonic transform pair on the DH sphere grid.
int plan_create(s2dw_plan_t* out, int L, int N, double lam, int J0, unsigned flags, bool sht_mode = false) {
  if (sht_mode) {
    N = 1;
    lam = 2.0;
    J0 = jmax_of(L, lam);
  }
  const int Jm = jmax_of(L, lam);
  if (J0 < 0 || J0 > Jm) return S2DW_EINVAL;
  const int J = Jm - J0;
  if (J + 1 > 64) return S2DW_ENOTSUP;
  s2dw_plan_s* p = new s2dw_plan_s();
  p->L = L;
  p->N = N;
  p->J0 = J0;
  p->J = J;
  p->nscale = J + 1;
  p->flags = flags | S2DW_REAL_SIGNAL;
  p->lam = lam;
  p->fp64 = (flags & S2DW_FP64) != 0;
  p->E = contract_rows_per_thread(p->fp64);
  p->TMP = 8 * p->E;
  cudaStream_t st = nullptr;
  double *kap = nullptr, *phi = nullptr, *sabs = nullptr, *q = nullptr, *gl = nullptr;
  double2* psi = nullptr;
  int rc = S2DW_OK;
  try {
    ck(cudaGetDevice(&p->device));
    setup_stream();  // configures the caching memory pool once per device
    ck(cudaStreamCreateWithFlags(&p->pst, cudaStreamNonBlocking));
    ck(cudaEventCreateWithFlags(&p->last_use, cudaEventDisableTiming));
    st = p->pst;
    std::vector<double> glx, glw;
    const int Q = 16, PAN = 32;
    gauss_legendre(Q, glx, glw);
    amalloc(&gl, (2 * Q + 1) * sizeof(double), st);  // nodes, weights, the kappa normalisation
    ck(cudaMemcpyAsync(gl, glx.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st));
    ck(cudaMemcpyAsync(gl + Q, glw.data(), Q * sizeof(double), cudaMemcpyHostToDevice, st));
    amalloc(&kap, (size_t)(J + 1) * L * sizeof(double), st);
    amalloc(&phi, (size_t)L * sizeof(double), st);
    amalloc(&sabs, (size_t)L * N * sizeof(double), st);
    amalloc(&psi, (size_t)(J + 1) * L * N * sizeof(double2), st);
    amalloc(&q, (size_t)2 * L * sizeof(double), st);
    ck(launch_kernel_values(kap, phi, sabs, psi, q, L, N, J, lam, gl, gl + Q, Q, PAN, gl + 2 * Q, st));
    std::vector<double> kap_h((size_t)(J + 1) * L);
    p->phi_host.resize(L);
    p->psi_host.resize((size_t)(J + 1) * L * N * 2);
    ck(cudaMemcpyAsync(kap_h.data(), kap, kap_h.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ck(cudaMemcpyAsync(p->phi_host.data(), phi, L * sizeof(double), cudaMemcpyDeviceToHost, st));
    ck(cudaMemcpyAsync(p->psi_host.data(), psi, p->psi_host.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
    ck(cudaStreamSynchronize(st));
    if (sht_mode) {
      for (int l = 0; l < L; ++l) p->phi_host[l] = std::sqrt((2.0 * l + 1.0) / (4.0 * 3.14159265358979323846));
      ck(cudaMemcpyAsync(phi, p->phi_host.data(), L * sizeof(double), cudaMemcpyHostToDevice, st));
      ck(cudaStreamSynchronize(st));
      p->nscale = 0;
      p->sht = true;
    }
    // supports where kappa^j(l) > 0 and their overlaps
    p->lo.assign(p->nscale, -1);
    p->hi.assign(p->nscale, -1);
    p->Lj.assign(p->nscale, 0);
    std::vector<int> count(L, 0);
    for (int j = 0; j < p->nscale; ++j)
      for (int l = 0; l < L; ++l)
        if (kap_h[(size_t)j * L + l] > 0.0) {
          if (p->lo[j] < 0) p->lo[j] = l;
          p->hi[j] = l;
          count[l]++;
        }
    for (int l = 0; l < L; ++l)
      if (count[l] > 2) throw CudaFail{cudaErrorInvalidValue};
    for (int j = 0; j < p->nscale; ++j) {
      if (p->hi[j] >= 0) p->Lj[j] = p->hi[j] + 1;
      if (j >= 2 && p->hi[j] >= 0 && p->lo[j - 2] >= 0 && p->lo[j - 2] <= p->hi[j])
        throw CudaFail{cudaErrorInvalidValue};
      p->lend_w = std::max(p->lend_w, p->hi[j]);
      p->L0 = std::max(p->L0, p->Lj[j]);
    }
    p->lphi = 0;
    for (int l = 0; l < L; ++l)
      if (p->phi_host[l] > 0.0) p->lphi = l;
    p->Lphi = p->lphi + 1;
    p->Ycols = p->Lj;
    p->Ycols.push_back(p->Lphi);
    p->Lp = round_up(L, 32);  // R-table row pitch: whole 32-row tiles are staged
    p->Lp32 = round_up(L, 32);
    p->Lphip = round_up(p->Lphi, 32);
    p->Lphip32 = round_up(p->Lphi, 32);
    p->nbr = (p->L0 + p->TMP - 1) / p->TMP;
    p->nbr_phi = (p->Lphi + p->TMP - 1) / p->TMP;
    // sampling grid of every scale (last: the scaling part): the full grid of
    // band-limit L, or with S2DW_MULTIRES the grid of the scale's own
    // band-limit (1 + the last l with a nonzero kernel)
    p->multires = (flags & S2DW_MULTIRES) != 0;
    p->mw = (flags & S2DW_MW) != 0;
    if (p->mw && p->multires) throw CudaFail{cudaErrorInvalidValue};
    std::vector<int> Lg(p->nscale + 1);
    for (int j = 0; j < p->nscale; ++j) Lg[j] = p->multires ? std::max(1, p->Lj[j]) : L;
    Lg[p->nscale] = p->multires ? p->Lphi : L;
    std::vector<int> uniq(Lg);
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    p->gt.resize(uniq.size());
    p->logM = 0;
    for (size_t g = 0; g < uniq.size(); ++g) {
      auto& G = p->gt[g];
      G.L = uniq[g];
      G.logM = 5;  // the radix-16 convolution engine needs M >= 32
      while ((1 << G.logM) < 4 * G.L - 2) ++G.logM;
      G.M = 1 << G.logM;
      G.nb = p->mw ? G.L : 2 * G.L;
      p->logM = std::max(p->logM, G.logM);
    }
    p->M = 1 << p->logM;
    p->grid_of.resize(p->nscale + 1);
    for (int j = 0; j <= p->nscale; ++j)
      p->grid_of[j] = (int)(std::lower_bound(uniq.begin(), uniq.end(), Lg[j]) - uniq.begin());
    p->woff.resize(p->nscale + 1);
    int64_t wacc = 0;
    for (int j = 0; j < p->nscale; ++j) {
      p->woff[j] = wacc;
      wacc += (int64_t)N * p->gt[p->grid_of[j]].nb * (2 * Lg[j] - 1);
    }
    p->woff[p->nscale] = wacc;
    p->tab = delta_acquire(L, st);
    if (p->fp64) plan_build_typed<double>(p, kap, phi, sabs, q, st);
    else plan_build_typed<float>(p, kap, phi, sabs, q, st);
    ck(cudaStreamSynchronize(st));
  } catch (const CudaFail& e) {
    rc = (e.err == cudaErrorMemoryAllocation) ? S2DW_ENOMEM
         : (e.err == cudaErrorInvalidValue) ? S2DW_EINVAL
                                             : S2DW_ECUDA;
  } catch (const std::bad_alloc&) {
    rc = S2DW_ENOMEM;
  } catch (...) {
    rc = S2DW_ECUDA;
  }
  if (st) {
    afree(gl, st);
    afree(kap, st);
    afree(phi, st);
    afree(sabs, st);
    afree(psi, st);
    afree(q, st);
  }
  if (rc != S2DW_OK) {
    cudaGetLastError();
    delete p;
    return rc;
  }
  *out = p;
  return S2DW_OK;
}

int err_of(cudaError_t e) {
  if (e == cudaSuccess) return S2DW_OK;
  if (e == cudaErrorMemoryAllocation) return S2DW_ENOMEM;
  return S2DW_ECUDA;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

const char* s2dw_strerror(int status) {
  switch (status) {
    case S2DW_OK: return "ok";
    case S2DW_EINVAL: return "invalid argument";
    case S2DW_ENOMEM: return "device allocation failed";
    case S2DW_ECUDA: return "CUDA call or kernel launch failed";
    case S2DW_ETIMEOUT: return "bounded device wait ran out";
    case S2DW_EBUSY: return "resource busy";
    case S2DW_ENOTSUP: return "not supported by this build";
    default: return "unknown status";
  }
}

int s2dw_plan(s2dw_plan_t* out, int L, int N, double lambda, int J0, unsigned flags) {
  if (!out) return S2DW_EINVAL;
  *out = nullptr;
  const unsigned prec = flags & (S2DW_FP64 | S2DW_MIXED);
  if (prec != S2DW_FP64 && prec != S2DW_MIXED) return S2DW_EINVAL;
  if (flags & ~(unsigned)(S2DW_FP64 | S2DW_MIXED | S2DW_REAL_SIGNAL | S2DW_MULTIRES | S2DW_MW)) return S2DW_EINVAL;
  if ((flags & S2DW_MW) && (flags & S2DW_MULTIRES)) return S2DW_EINVAL;
  // invalid requests (no transform exists) before limits of this build
  if (L < 2 || N < 1 || N > L) return S2DW_EINVAL;
  if (!(lambda > 1.0) || !std::isfinite(lambda)) return S2DW_EINVAL;
  const int jm = jmax_of(L, lambda);
  if (jm < 0) return S2DW_ENOTSUP;  // over a million scales
  if (J0 < 0 || J0 > jm) return S2DW_EINVAL;
  if (L > 2048 || N > 8) return S2DW_ENOTSUP;
  try {
    return plan_create(out, L, N, lambda, J0, flags);
  } catch (...) {
    return S2DW_ECUDA;
  }
}

int s2dw_plan_destroy(s2dw_plan_t plan) {
  if (!plan) return S2DW_OK;
  drop_batches_with(plan);
  delete plan;  // waits for the plan's last recorded call, frees stream-ordered
  return err_of(cudaGetLastError());
}

int s2dw_query(s2dw_plan_t p, int* J, int64_t* w_elems_per_scale, int64_t* wphi_elems, int64_t* workspace_bytes,
               int64_t* total_device_bytes) {
  if (!p) return S2DW_EINVAL;
  const int64_t L = p->L, n = 2 * L - 1;
  const int64_t wps = p->multires ? 0 : (int64_t)p->N * p->gt[0].nb * n;
  const auto& Gp = p->gt[p->grid_of[p->nscale]];
  const int64_t Lp = Gp.L, wph = (int64_t)Gp.nb * (2 * Lp - 1);
  const int64_t el = p->fp64 ? 8 : 4;
  if (J) *J = p->J;
  if (w_elems_per_scale) *w_elems_per_scale = wps;
  if (wphi_elems) *wphi_elems = wph;
  if (workspace_bytes) *workspace_bytes = (int64_t)p->ws_bytes;
  if (total_device_bytes)
    *total_device_bytes = (int64_t)p->ws_bytes + (p->woff[p->nscale] + wph) * el + L * L * 2 * el;
  return S2DW_OK;
}

int s2dw_steer(s2dw_plan_t p, const void* W, const double* gammas, int ngamma, void* out, void* stream) {
  if (!p || !W || !gammas || !out || ngamma < 1 || ngamma > kSteerMaxGamma) return S2DW_EINVAL;
  const int N = p->N;
  SteerWeights sw;
  std::memset(&sw, 0, sizeof(sw));
  for (int t = 0; t < ngamma; ++t)
    for (int g = 0; g < N; ++g) {
      const double x = gammas[t] - 3.14159265358979323846 * g / N;
      double z = 0.0;
      for (int k = 0; k < N; ++k) z += std::cos((-(N - 1) + 2 * k) * x);
      sw.w[t][g] = z / N;
    }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const size_t el = p->fp64 ? sizeof(double) : sizeof(float);
  cudaError_t e = cudaSuccess;
  if (!p->multires) {
    const int64_t per_scale = (int64_t)p->gt[0].nb * (2 * p->L - 1);
    e = p->fp64 ? launch_steer<double>(W, out, sw, p->nscale, N, ngamma, per_scale, st)
                : launch_steer<float>(W, out, sw, p->nscale, N, ngamma, per_scale, st);
  } else {
    // scales of different grids: out holds [ngamma][2Lg][2Lg-1] per scale, in order
    for (int j = 0; j < p->nscale && e == cudaSuccess; ++j) {
      const int64_t Lg = p->gt[p->grid_of[j]].L, per_scale = 2 * Lg * (2 * Lg - 1);
      const char* Wj = reinterpret_cast<const char*>(W) + (size_t)p->woff[j] * el;
      char* Oj = reinterpret_cast<char*>(out) + (size_t)(p->woff[j] / N) * ngamma * el;
      e = p->fp64 ? launch_steer<double>(Wj, Oj, sw, 1, N, ngamma, per_scale, st)
                  : launch_steer<float>(Wj, Oj, sw, 1, N, ngamma, per_scale, st);
    }
  }
  return err_of(e);
}

namespace {
int sht_child(s2dw_plan_t p, s2dw_plan_t* c) {
  if (!p->sht_child) {
    const int rc = plan_create(&p->sht_child, p->L, 1, 2.0, 0, p->fp64 ? S2DW_FP64 : S2DW_MIXED, true);
    if (rc != S2DW_OK) {
      p->sht_child = nullptr;
      return rc;
    }
  }
  *c = p->sht_child;
  return S2DW_OK;
}
}  // namespace

int s2dw_sht_inverse(s2dw_plan_t p, const void* flm, void* fpix, void* stream) {
  if (!p || !flm || !fpix) return S2DW_EINVAL;
  s2dw_plan_t c = nullptr;
  const int rc = sht_child(p, &c);
  if (rc != S2DW_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  ptrs.f[0] = flm;
  ptrs.Wphi[0] = fpix;
  if (c->fp64) run_analysis<double>(c->own, ptrs, st);
  else run_analysis<float>(c->own, ptrs, st);
  mark_use(c, st);
  return err_of(cudaGetLastError());
}

int s2dw_sht_forward(s2dw_plan_t p, const void* fpix, void* flm, void* stream) {
  if (!p || !flm || !fpix) return S2DW_EINVAL;
  s2dw_plan_t c = nullptr;
  const int rc = sht_child(p, &c);
  if (rc != S2DW_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  ptrs.Wphi[0] = const_cast<void*>(fpix);
  ReduceJobs rj;
  std::memset(&rj, 0, sizeof(rj));
  rj.dw[0] = c->own.desc_w;
  rj.dp[0] = c->own.desc_phi;
  rj.out[0] = flm;
  rj.L[0] = c->L;
  rj.lend[0] = c->lend_w;
  rj.Lphi[0] = c->Lphi;
  rj.sht[0] = 1;
  if (c->fp64) run_synthesis<double>(c->own, ptrs, rj, 1, st);
  else run_synthesis<float>(c->own, ptrs, rj, 1, st);
  mark_use(c, st);
  return err_of(cudaGetLastError());
}

int s2dw_scale_grid(s2dw_plan_t p, int j, int* Lgrid, int64_t* offset, int64_t* elems) {
  if (!p || j < 0 || j > p->nscale) return S2DW_EINVAL;
  const int64_t Lg = p->gt[p->grid_of[j]].L, nb = p->gt[p->grid_of[j]].nb;
  const int64_t per = (j == p->nscale ? 1 : p->N) * nb * (2 * Lg - 1);
  if (Lgrid) *Lgrid = (int)Lg;
  if (offset) *offset = (j == p->nscale) ? 0 : p->woff[j];
  if (elems) *elems = per;
  return S2DW_OK;
}

int s2dw_alpha_method(s2dw_plan_t p, int j, int dir, int* method, int* fft_len, int* segments, int* seg_len) {
  if (!p || j < 0 || j > p->nscale || dir < 0 || dir > 1) return S2DW_EINVAL;
  const int Lj = p->Ycols[j];
  const auto& G = p->gt[p->grid_of[j]];
  const auto& sgt = p->seg[j];
  int m = 1, len = G.M, ns = 1, sl = 2 * G.L - 1;
  (void)Lj;
  if (p->alpha_mode[dir][j] == 0) {
    m = 0;
    len = ns = sl = 0;
  } else if (p->alpha_mode[dir][j] == 2) {
    m = 2;
    len = 1 << sgt.logM;
    ns = sgt.S;
    sl = sgt.P;
  }
  if (method) *method = m;
  if (fft_len) *fft_len = len;
  if (segments) *segments = ns;
  if (seg_len) *seg_len = sl;
  return S2DW_OK;
}

// ---- launch methods and the autotuner -------------------------------------
static int choices_count(s2dw_plan_t p) { return 3 + 2 * (p->nscale + 1); }

// Whether method v is available for choice idx of the plan (layout of s2dw_plan_choices).
static bool choice_valid(s2dw_plan_t p, int idx, int v) {
  if (idx < 2) return v == 0 || v == 1;  // grids without half-length transforms keep the FFT
  if (idx == choices_count(p) - 1) {  // contraction CTA shape (FP32 plans with N <= 5 have three)
    if (p->fp64) return v == 0;
    return pair_two_tiles(p->N) ? (v >= kPairShapePair && v <= kPairShapeTile2) : v == kPairShapeTile;
  }
  const int j = (idx - 2) / 2, d = (idx - 2) % 2;
  const int Lj = p->Ycols[j];
  if (v == 0) return Lj <= (d == 0 ? kDirectMaxLjAna : kDirectMaxLj);  // direct kernels sized for L_j <= 32
  if (v == 1) return true;
  if (v == 2) return p->seg[j].S > 0;  // segment tables built at plan creation
  return false;
}

static void choices_get(s2dw_plan_t p, int* c) {
  c[0] = p->beta_mode[0];
  c[1] = p->beta_mode[1];
  for (int j = 0; j <= p->nscale; ++j) {
    c[2 + 2 * j] = p->alpha_mode[0][j];
    c[3 + 2 * j] = p->alpha_mode[1][j];
  }
  c[choices_count(p) - 1] = p->fp64 ? 0 : p->pair_shape;
}

static void choices_put(s2dw_plan_t p, const int* c) {
  p->beta_mode[0] = c[0];
  p->beta_mode[1] = c[1];
  for (int j = 0; j <= p->nscale; ++j) {
    p->alpha_mode[0][j] = c[2 + 2 * j];
    p->alpha_mode[1][j] = c[3 + 2 * j];
  }
  if (!p->fp64) {
    const int shape = c[choices_count(p) - 1];
    if (shape != p->pair_shape) {
      p->pair_shape = shape;
      build_pair_tasks(p->L0, p->lend_w, shape == kPairShapePair, p->tab->Lmax, p->ptasks_w_host);
    }
  }
  drop_batches_with(p);
  if (p->fp64) own_lists_build<double>(p);
  else own_lists_build<float>(p);
}

int s2dw_plan_choices(s2dw_plan_t p, int* choices, int* n) {
  if (!p || !n) return S2DW_EINVAL;
  const int need = choices_count(p);
  if (!choices) {
    *n = need;
    return S2DW_OK;
  }
  if (*n < need) {
    *n = need;
    return S2DW_EINVAL;
  }
  choices_get(p, choices);
  *n = need;
  return S2DW_OK;
}

int s2dw_plan_set_choices(s2dw_plan_t p, const int* choices, int n) {
  if (!p || !choices || n != choices_count(p)) return S2DW_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!choice_valid(p, i, choices[i])) return S2DW_EINVAL;
  try {
    ck(cudaEventSynchronize(p->last_use));  // this plan's calls so far (the lists are replaced)
    choices_put(p, choices);
    ck(cudaStreamSynchronize(p->pst));
  } catch (const CudaFail& e) {
    return err_of(e.err);
  } catch (...) {
    return S2DW_ECUDA;
  }
  return S2DW_OK;
}

int s2dw_plan_tune(s2dw_plan_t p, int reps, int* choices, int* n) {
  if (!p || reps < 1 || reps > 64 || (choices && !n)) return S2DW_EINVAL;
  const int nc = choices_count(p);
  if (choices && *n < nc) {
    *n = nc;
    return S2DW_EINVAL;
  }
  cudaStream_t st = p->pst;
  const size_t el = p->fp64 ? 8 : 4;
  int64_t wphi = 0;
  s2dw_query(p, nullptr, nullptr, &wphi, nullptr, nullptr);
  const size_t fbytes = (size_t)p->L * p->L * 2 * el;
  const size_t wbytes = ((size_t)p->woff[p->nscale] + (size_t)wphi) * el;
  void *f = nullptr, *fr = nullptr, *W = nullptr;
  constexpr int A = s2dw_plan_s::kEvAna, S = s2dw_plan_s::kEvSyn;
  cudaEvent_t ev[A + S] = {};
  std::vector<int> cur(nc), best(nc);
  try {
    ck(cudaEventSynchronize(p->last_use));
    amalloc(&f, fbytes, st);
    amalloc(&fr, fbytes, st);
    amalloc(&W, wbytes, st);
    // nonzero inputs: the analysis then writes W of the same kind for the synthesis
    if (p->fp64) ck(launch_fill_noise<double>(reinterpret_cast<double*>(f), (int64_t)(fbytes / 8), 0x5eedu, st));
    else ck(launch_fill_noise<float>(reinterpret_cast<float*>(f), (int64_t)(fbytes / 4), 0x5eedu, st));
    ck(cudaMemsetAsync(W, 0, wbytes, st));
    for (auto& e : ev) ck(cudaEventCreate(&e));
    CallPtrs ptrs;
    std::memset(&ptrs, 0, sizeof(ptrs));
    ptrs.f[0] = f;
    ptrs.out[0] = fr;
    ptrs.W[0] = W;
    ptrs.Wphi[0] = reinterpret_cast<char*>(W) + (size_t)p->woff[p->nscale] * el;
    // milliseconds of the beta launch and of the alpha launches of each
    // direction, the minimum over `reps` round trips
    auto measure = [&](double (&ms)[5]) {
      for (double& v : ms) v = 1e30;
      for (int r = 0; r < reps; ++r) {
        ReduceJobs rj;
        std::memset(&rj, 0, sizeof(rj));
        rj.dw[0] = p->own.desc_w;
        rj.dp[0] = p->own.desc_phi;
        rj.out[0] = fr;
        rj.L[0] = p->L;
        rj.lend[0] = p->lend_w;
        rj.Lphi[0] = p->Lphi;
        if (p->fp64) {
          run_analysis<double>(p->own, ptrs, st, ev);
          run_synthesis<double>(p->own, ptrs, rj, 1, st, ev + A);
        } else {
          run_analysis<float>(p->own, ptrs, st, ev);
          run_synthesis<float>(p->own, ptrs, rj, 1, st, ev + A);
        }
        ck(cudaGetLastError());
        ck(cudaEventSynchronize(ev[A + S - 1]));
        float t[6] = {};
        ck(cudaEventElapsedTime(&t[0], ev[2], ev[3]));          // analysis beta
        ck(cudaEventElapsedTime(&t[1], ev[A + 3], ev[A + 4]));  // synthesis beta
        ck(cudaEventElapsedTime(&t[2], ev[3], ev[6]));          // analysis alpha (all launches)
        ck(cudaEventElapsedTime(&t[3], ev[A + 0], ev[A + 3]));  // synthesis alpha
        ck(cudaEventElapsedTime(&t[4], ev[0], ev[2]));          // analysis contractions
        ck(cudaEventElapsedTime(&t[5], ev[A + 4], ev[A + 6]));  // synthesis contractions
        t[4] += t[5];
        for (int i = 0; i < 5; ++i) ms[i] = std::min(ms[i], (double)t[i]);
      }
    };
    // the choices now in place beat the incumbent's time base[i] on stage i:
    // 3 % faster in a first measurement and again in a second one (the
    // incumbent re-measured between them), so that noise does not switch methods
    auto better = [&](double (&ms)[5], int i, double (&base)[5]) {
      measure(ms);
      if (!(ms[i] < 0.97 * base[i])) return false;
      std::vector<int> trial(nc);
      choices_get(p, trial.data());
      choices_put(p, cur.data());
      double again[5];
      measure(again);
      base[i] = std::min(base[i], again[i]);
      choices_put(p, trial.data());
      double ms2[5];
      measure(ms2);
      for (int k = 0; k < 5; ++k) ms[k] = std::min(ms[k], ms2[k]);
      return ms[i] < 0.97 * base[i];
    };
    choices_get(p, cur.data());
    double base[5];
    choices_put(p, cur.data());
    measure(base);  // warms up as well
    measure(base);
    // coordinate descent: the beta method of each direction, then each
    // scale's alpha method (largest band first) against its direction's total
    for (int d = 0; d < 2; ++d) {
      for (int v = 0; v < 2; ++v) {
        if (v == cur[d] || !choice_valid(p, d, v)) continue;
        std::vector<int> trial(cur);
        trial[d] = v;
        choices_put(p, trial.data());
        double ms[5];
        if (better(ms, d, base)) {
          cur = trial;
          base[d] = ms[d];
        }
      }
    }
    choices_put(p, cur.data());
    measure(base);
    std::vector<int> order(p->nscale + 1);
    for (int j = 0; j <= p->nscale; ++j) order[j] = j;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return p->Ycols[a] > p->Ycols[b]; });
    for (int d = 0; d < 2; ++d)
      for (int j : order) {
        const int idx = 2 + 2 * j + d;
        for (int v = 0; v < 3; ++v) {
          if (v == cur[idx] || !choice_valid(p, idx, v) || p->Ycols[j] <= 0) continue;
          std::vector<int> trial(cur);
          trial[idx] = v;
          choices_put(p, trial.data());
          double ms[5];
          if (better(ms, 2 + d, base)) {
            cur = trial;
            base[2 + d] = ms[2 + d];
          }
        }
      }
    // the contraction's CTA shape (both directions)
    {
      const int idx = nc - 1;
      for (int v = 0; v < 3; ++v) {
        if (v == cur[idx] || !choice_valid(p, idx, v)) continue;
        std::vector<int> trial(cur);
        trial[idx] = v;
        choices_put(p, trial.data());
        double ms[5];
        if (better(ms, 4, base)) {
          cur = trial;
          base[4] = ms[4];
        }
      }
    }
    choices_put(p, cur.data());
    ck(cudaStreamSynchronize(st));
  } catch (const CudaFail& e) {
    cudaStreamSynchronize(st);
    for (auto& e2 : ev) if (e2) cudaEventDestroy(e2);
    afree(f, st);
    afree(fr, st);
    afree(W, st);
    return err_of(e.err);
  } catch (...) {
    cudaStreamSynchronize(st);
    for (auto& e2 : ev) if (e2) cudaEventDestroy(e2);
    afree(f, st);
    afree(fr, st);
    afree(W, st);
    return S2DW_ECUDA;
  }
  for (auto& e : ev) cudaEventDestroy(e);
  afree(f, st);
  afree(fr, st);
  afree(W, st);
  cudaStreamSynchronize(st);
  if (choices) {
    choices_get(p, choices);
    *n = nc;
  }
  return S2DW_OK;
}

int s2dw_wait_timeouts(int* count) {
  if (!count) return S2DW_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return err_of(e);
  e = alpha_tc_timeouts(count);
  if (e != cudaSuccess) return err_of(e);
  int pc = 0;
  e = pair_timeouts(&pc);
  if (e != cudaSuccess) return err_of(e);
  *count += pc;
  return *count > 0 ? S2DW_ETIMEOUT : S2DW_OK;
}

int s2dw_wait_probe(long long limit_cycles, void* stream) {
  const long long lim = std::min(std::max(limit_cycles, 1000LL), 2000000000LL);
  return err_of(alpha_tc_wait_probe(lim, reinterpret_cast<cudaStream_t>(stream)));
}

int s2dw_launch_counts(s2dw_plan_t p, int* analysis, int* synthesis) {
  if (!p) return S2DW_EINVAL;
  const Lists& ls = p->own;
  int contract = ls.ntiles_phi > 0 ? 1 : 0;
  for (auto& t : ls.tiles_w) contract += t.second.second > 0 ? 1 : 0;
  auto has = [&](int k) {
    if (k >= CZT_BETA_ANA_DCT && k <= CZT_BETA_RS_DCT) return (int)ls.dct_parts[k - CZT_BETA_ANA_DCT].size();
    return ls.items[k] > 0 ? 1 : 0;
  };
  const int fpack = (!p->fp64 && ls.njobs > 0 && ls.nbmax > 0) ? 1 : 0;  // f packing of the FP32 contraction
  if (analysis) *analysis = fpack + contract + has(0) + has(1) + has(4) + has(6) + has(8) + has(13);
  if (synthesis)
    *synthesis = contract + has(2) + has(3) + has(5) + has(7) + has(9) + has(10) + has(11) + has(12) + has(14) +
                 has(15) + 1;
  return S2DW_OK;
}

int s2dw_kernels(s2dw_plan_t p, double* psi, double* phi) {
  if (!p) return S2DW_EINVAL;
  if (psi) std::memcpy(psi, p->psi_host.data(), p->psi_host.size() * sizeof(double));
  if (phi) std::memcpy(phi, p->phi_host.data(), p->phi_host.size() * sizeof(double));
  return S2DW_OK;
}

int s2dw_analysis(s2dw_plan_t p, const void* flm, void* W, void* Wphi, void* stream) {
  if (!p || !flm || !W || !Wphi) return S2DW_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  ptrs.f[0] = flm;
  ptrs.W[0] = W;
  ptrs.Wphi[0] = Wphi;
  cudaEvent_t* ev = nullptr;
  if (p->prof && p->nana < s2dw_plan_s::kProfCalls && !capturing(st))
    ev = p->ev_ana.data() + s2dw_plan_s::kEvAna * (p->nana++);
  if (p->fp64) run_analysis<double>(p->own, ptrs, st, ev);
  else run_analysis<float>(p->own, ptrs, st, ev);
  mark_use(p, st);
  return err_of(cudaGetLastError());
}

int s2dw_synthesis(s2dw_plan_t p, const void* W, const void* Wphi, void* flm, void* stream) {
  if (!p || !flm || !W || !Wphi) return S2DW_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  ptrs.out[0] = flm;
  ptrs.W[0] = const_cast<void*>(W);
  ptrs.Wphi[0] = const_cast<void*>(Wphi);
  ReduceJobs rj;
  std::memset(&rj, 0, sizeof(rj));
  rj.dw[0] = p->own.desc_w;
  rj.dp[0] = p->own.desc_phi;
  rj.out[0] = flm;
  rj.L[0] = p->L;
  rj.lend[0] = p->lend_w;
  rj.Lphi[0] = p->Lphi;
  cudaEvent_t* ev = nullptr;
  if (p->prof && p->nsyn < s2dw_plan_s::kProfCalls && !capturing(st))
    ev = p->ev_syn.data() + s2dw_plan_s::kEvSyn * (p->nsyn++);
  if (p->fp64) run_synthesis<double>(p->own, ptrs, rj, 1, st, ev);
  else run_synthesis<float>(p->own, ptrs, rj, 1, st, ev);
  mark_use(p, st);
  return err_of(cudaGetLastError());
}

int s2dw_profile(s2dw_plan_t p, int enable) {
  if (!p) return S2DW_EINVAL;
  if (enable && p->ev_ana.empty()) {
    p->ev_ana.assign(s2dw_plan_s::kEvAna * s2dw_plan_s::kProfCalls, nullptr);
    p->ev_syn.assign(s2dw_plan_s::kEvSyn * s2dw_plan_s::kProfCalls, nullptr);
    for (auto& e : p->ev_ana)
      if (cudaEventCreate(&e) != cudaSuccess) return S2DW_ECUDA;
    for (auto& e : p->ev_syn)
      if (cudaEventCreate(&e) != cudaSuccess) return S2DW_ECUDA;
  }
  p->prof = enable != 0;
  p->nana = 0;
  p->nsyn = 0;
  return S2DW_OK;
}

int s2dw_profile_read(s2dw_plan_t p, double* ms, int* ncalls) {
  if (!p || !ms) return S2DW_EINVAL;
  constexpr int A = s2dw_plan_s::kEvAna, S = s2dw_plan_s::kEvSyn;
  for (int i = 0; i < A + S - 2; ++i) ms[i] = 0.0;
  if (ncalls) ncalls[0] = ncalls[1] = 0;
  if (p->ev_ana.empty()) return S2DW_OK;
  cudaError_t e = cudaSuccess;
  int na = 0, ns = 0;
  for (int c = 0; c < p->nana; ++c) {
    cudaEvent_t* ev = p->ev_ana.data() + A * c;
    if ((e = cudaEventSynchronize(ev[A - 1])) != cudaSuccess) return err_of(e);
    for (int i = 0; i < A - 1; ++i) {
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, ev[i], ev[i + 1])) != cudaSuccess) return err_of(e);
      ms[i] += t;
    }
    ++na;
  }
  for (int c = 0; c < p->nsyn; ++c) {
    cudaEvent_t* ev = p->ev_syn.data() + S * c;
    if ((e = cudaEventSynchronize(ev[S - 1])) != cudaSuccess) return err_of(e);
    for (int i = 0; i < S - 1; ++i) {
      float t = 0.f;
      if ((e = cudaEventElapsedTime(&t, ev[i], ev[i + 1])) != cudaSuccess) return err_of(e);
      ms[A - 1 + i] += t;
    }
    ++ns;
  }
  if (ncalls) {
    ncalls[0] = na;
    ncalls[1] = ns;
  }
  return S2DW_OK;
}

// Looks up (or builds) the launch lists of a plan set; g_batch_mu must be held
// by the caller until the launches using the entry are queued and recorded.
static int batch_lists(const s2dw_plan_t* plans, int njobs, BatchEnt** out, bool* fp64) {
  if (!plans || njobs < 1 || njobs > MAXB) return S2DW_EINVAL;
  std::vector<s2dw_plan_t> key(plans, plans + njobs);
  for (int i = 0; i < njobs; ++i) {
    if (!key[i]) return S2DW_EINVAL;
    for (int k = 0; k < i; ++k)
      if (key[k] == key[i]) return S2DW_EINVAL;
    if (key[i]->fp64 != key[0]->fp64) return S2DW_ENOTSUP;
  }
  *fp64 = key[0]->fp64;
  auto it = g_batch_cache.find(key);
  if (it == g_batch_cache.end()) {
    evict_batches();
    BatchEnt e;
    try {
      e.ls = *fp64 ? build_lists<double>(key) : build_lists<float>(key);
    } catch (const CudaFail& err) {
      return err_of(err.err);
    } catch (...) {
      return S2DW_ENOMEM;
    }
    if (cudaEventCreateWithFlags(&e.done, cudaEventDisableTiming) != cudaSuccess) {
      delete e.ls;
      return S2DW_ECUDA;
    }
    it = g_batch_cache.emplace(key, e).first;
  }
  it->second.tick = ++g_batch_tick;
  *out = &it->second;
  return S2DW_OK;
}

static void batch_used(BatchEnt* e, cudaStream_t st) {
  if (capturing(st)) e->pinned = true;
  else cudaEventRecord(e->done, st);
}

int s2dw_analysis_batch(const s2dw_plan_t* plans, const void* const* flm, void* const* W, void* const* Wphi,
                        int njobs, void* stream) {
  if (!flm || !W || !Wphi) return S2DW_EINVAL;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchEnt* be = nullptr;
  bool fp64 = false;
  int rc = batch_lists(plans, njobs, &be, &fp64);
  if (rc != S2DW_OK) return rc;
  const Lists* ls = be->ls;
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  for (int i = 0; i < njobs; ++i) {
    if (!flm[i] || !W[i] || !Wphi[i]) return S2DW_EINVAL;
    ptrs.f[i] = flm[i];
    ptrs.W[i] = W[i];
    ptrs.Wphi[i] = Wphi[i];
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fp64) run_analysis<double>(*ls, ptrs, st);
  else run_analysis<float>(*ls, ptrs, st);
  batch_used(be, st);
  for (int i = 0; i < njobs; ++i) mark_use(plans[i], st);
  return err_of(cudaGetLastError());
}

int s2dw_synthesis_batch(const s2dw_plan_t* plans, const void* const* W, const void* const* Wphi, void* const* flm,
                         int njobs, void* stream) {
  if (!flm || !W || !Wphi) return S2DW_EINVAL;
  std::lock_guard<std::mutex> lk(g_batch_mu);
  BatchEnt* be = nullptr;
  bool fp64 = false;
  int rc = batch_lists(plans, njobs, &be, &fp64);
  if (rc != S2DW_OK) return rc;
  const Lists* ls = be->ls;
  CallPtrs ptrs;
  std::memset(&ptrs, 0, sizeof(ptrs));
  ReduceJobs rj;
  std::memset(&rj, 0, sizeof(rj));
  const size_t dsz = fp64 ? sizeof(ContractDesc<double>) : sizeof(ContractDesc<float>);
  for (int i = 0; i < njobs; ++i) {
    if (!flm[i] || !W[i] || !Wphi[i]) return S2DW_EINVAL;
    ptrs.out[i] = flm[i];
    ptrs.W[i] = const_cast<void*>(W[i]);
    ptrs.Wphi[i] = const_cast<void*>(Wphi[i]);
    rj.dw[i] = reinterpret_cast<const char*>(ls->desc_w) + i * dsz;
    rj.dp[i] = reinterpret_cast<const char*>(ls->desc_phi) + i * dsz;
    rj.out[i] = flm[i];
    rj.L[i] = plans[i]->L;
    rj.lend[i] = plans[i]->lend_w;
    rj.Lphi[i] = plans[i]->Lphi;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fp64) run_synthesis<double>(*ls, ptrs, rj, njobs, st);
  else run_synthesis<float>(*ls, ptrs, rj, njobs, st);
  batch_used(be, st);
  for (int i = 0; i < njobs; ++i) mark_use(plans[i], st);
  return err_of(cudaGetLastError());
}

int s2dw_scale_support(s2dw_plan_t p, int j, int* lo, int* hi) {
  if (!p || j < 0 || j > p->nscale) return S2DW_EINVAL;
  if (j == p->nscale) {
    if (lo) *lo = 0;
    if (hi) *hi = p->lphi;
  } else {
    if (lo) *lo = p->lo[j];
    if (hi) *hi = p->hi[j];
  }
  return S2DW_OK;
}

int s2dw_delta_slab(s2dw_plan_t p, int l, double* host_out) {
  if (!p || !host_out || l < 0 || l >= p->L) return S2DW_EINVAL;
  const int64_t sz = delta_slab_size(l);
  std::vector<double> slab(sz);
  cudaError_t e = cudaMemcpy(slab.data(), p->tab->d64 + delta_slab_offset(l), sz * sizeof(double),
                             cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return err_of(e);
  for (int mp = 0; mp <= l; ++mp)
    for (int m = 0; m <= l; ++m) {
      double v;
      if (m >= 4 * (mp >> 2)) v = slab[delta_entry(l, mp, m)];
      else v = (((mp - m) & 1) ? -1.0 : 1.0) * slab[delta_entry(l, m, mp)];
      host_out[(size_t)mp * (l + 1) + m] = v;
    }
  return S2DW_OK;
}

int s2dw_stage(s2dw_plan_t p, int stage, int j, void* host_out, int64_t* nbytes) {
  if (!p || j < 0 || j > p->nscale || stage < 0 || stage > 1) return S2DW_EINVAL;
  const int Nj = (j == p->nscale) ? 1 : p->N;
  const int Lj = p->Ycols[j];
  const int64_t el = p->fp64 ? 16 : 8;
  const int64_t Lg = p->gt[p->grid_of[j]].L;  // the scale's beta grid
  const int64_t bytes = (stage == 0 ? (int64_t)Nj * Lj * Lj : (int64_t)Nj * 2 * Lg * Lj) * el;
  if (nbytes) *nbytes = bytes;
  if (!host_out) return S2DW_OK;
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return err_of(e);
  e = cudaMemcpy(host_out, stage == 0 ? p->Y[j] : p->X[j], bytes, cudaMemcpyDeviceToHost);
  return err_of(e);
}

}  // extern "C"
