// Fused l-contraction on tile pairs, FP32 (Sec. 3.2 Eq. (27); Sec. 3.3
// Eqs. (34), (32)); the same sums as contract.cuh:
//   analysis  G^j_{m'mk} = sum_{l in supp j} Delta^l_{m'm} f_lm R^j_{l m' k},
//             then the gamma step (Eq. (28)) as an epilogue into Y^j_g[m][m'];
//   synthesis partial_l(m) = sum_{m' in tile} Delta^l_{m'm} sum_{j,k} R^j_{l m' k} H^j_{m'mk},
//             H from Vhat by the gamma quadrature (Eq. (39)) as a prologue.
//
// What differs from contract.cuh is how Delta reaches the arithmetic.
// * Pair table.  For every pair of 32-wide blocks p <= q (m' block p, m
//   block q) the table stores, for l = 32q .. Lmax-1 one after the other, the
//   32 x 32 block D_l[r][c] = Delta^l_{32p+r, 32q+c} (zero where an index
//   exceeds l; a diagonal block holds both triangles).  One l of one tile is
//   one contiguous 4 KB run, and all l of a tile are one run, so a pipeline
//   stage is a single 1-D bulk copy (cp.async.bulk) issued by one thread.
// * Both tiles of a pair in one CTA.  Delta^l_{m'm} = (-1)^{m'-m}
//   Delta^l_{m m'}, so the block of pair (p, q) also serves the tile (q, p),
//   read transposed.  The sign is constant over l: it is applied to G in the
//   analysis epilogue and to H in the synthesis prologue.  Each Delta block is
//   read from HBM once per transform instead of twice.
// * R rows and f values are stored per 32-block with l outermost
//   (RSp[b][l][slot][n_k >= 0][32], fP[b][l][32]), so they too are one
//   contiguous run per stage and half.
// The ring of three or four stages (4 or 8 l each) is filled with cp.async by all
// threads (each owns fixed 16-byte chunks of a stage; measured faster here
// than one thread issuing 1-D bulk copies), which signal the stage's `full`
// mbarrier through cp.async.mbarrier.arrive; every warp arrives on the
// stage's `empty` mbarrier once it has read it, and the threads refill the
// slot one or two stages later.  Stages that lie inside one l-segment (constant
// scales in both accumulator slots) take a path without any checks; segment
// changes and the last stage take a slower one.  Every wait is bounded
// (about a second): a CTA that gives up stops computing, waits for its own
// copies and counts the event for s2dw_wait_timeouts.
//
// Thread layout: HALVES * 256 threads; half h computes tile A = (p, q) (h = 0)
// or tile B = (q, p) (h = 1), each thread E = 4 consecutive rows m' and one
// column m.  Tile A maps lanes along m (its 4 Delta values are 4 scalar
// loads from distinct banks), tile B maps lanes along row groups (its 4
// values are one 16-byte load D_l[c][4g..4g+3], 8 distinct bank groups per
// quarter warp).  HALVES = 1 (N > 5, whose accumulators need more than 128
// registers) launches one CTA per tile; a task then names its half.
#pragma once

#include <type_traits>

#include "contract.cuh"
#include "tc.cuh"

namespace s2dw {

// Ring geometry (PairGeom): eight l per stage in the tile-pair CTAs, four
// in the one-tile CTAs; four stages, three in the tile-pair synthesis, whose
// partial sums take the rest of the shared memory; a slot is refilled two
// stages after it was read (one in that synthesis).  Measured at L = 1024,
// N = 5 (analysis / synthesis, ms per launch): two l per stage 0.55 / 0.56;
// four 0.46 / 0.46; eight in the analysis 0.45; with the packed builtins
// 0.40 / 0.45; eight in the synthesis (three stages) 0.40 / 0.39.  Refills
// one or three stages after the read were slower (0.50 and 0.79 ms in the
// four-l analysis, 0.49 ms in the three-stage synthesis at two).  The
// waits, arrivals and refills of a stage are paid once per stage.
constexpr int kPairKLMax = 8;    // l per pipeline stage, at most (tables are padded for it)

__device__ int g_pair_timeouts;  // bounded waits that gave up (read and reset by the host)

template <int N, int NSLOT, bool SYN, int HALVES>
struct PairGeom {
  static constexpr int NH = (N + 1) / 2;
  static constexpr int RROW = NSLOT * NH * 32;   // floats of one l of one R block
  static constexpr int DP = 36;                  // shared-memory pitch of a Delta row (32 + 4)
  static constexpr int DL = 32 * DP;             // floats of one l of Delta in shared memory
  static constexpr int KL = HALVES == 1 ? 4 : 8;  // l per stage (even: a position's parity is its l's)
  static constexpr int STAGES = (SYN && HALVES == 2) ? 3 : 4;  // ring depth
  static constexpr int LAG = (SYN && HALVES == 2) ? 1 : 2;     // refill this many stages after the read
  static constexpr int D_F = KL * DL;            // Delta floats per stage
  static constexpr int R_F = KL * RROW;          // R floats per stage and half
  static constexpr int F_F = SYN ? 0 : KL * 64;  // f floats per stage and half
  static constexpr int R_OFF = D_F;
  static constexpr int F_OFF = R_OFF + HALVES * R_F;
  static constexpr int SIZE = F_OFF + HALVES * F_F;
  static constexpr size_t BYTES = (size_t)SIZE * 4;
  // synthesis partials per (buffer, l, half): [row group][32 columns]
  static constexpr int RED_SLAB = 8 * 32;
  static constexpr size_t RED_BYTES = SYN ? (size_t)2 * LCH * HALVES * RED_SLAB * sizeof(float2) : 0;
  static constexpr size_t SMEM = STAGES * BYTES + RED_BYTES;
};

// Accumulators of rows (2i, 2i+1) as float2 pairs for the packed FP32
// builtins (__ffma2_rn); the tile-pair CTAs use these (measured: analysis
// 0.451 -> 0.399 ms at L = 1024, N = 5), the one-tile CTAs the inline-PTX
// f32x2 forms of Acc<float, ..., true>, with which they do not spill
template <int E, int NSLOT, int N>
struct AccF2 {
  float2 x[E / 2][NSLOT][N], y[E / 2][NSLOT][N];
  __device__ __forceinline__ cx<float> get(int e, int s, int k) const {
    const float2 a = x[e >> 1][s][k], b = y[e >> 1][s][k];
    return (e & 1) ? mkc<float>(a.y, b.y) : mkc<float>(a.x, b.x);
  }
  __device__ __forceinline__ void set(int e, int s, int k, cx<float> v) {
    if (e & 1) {
      x[e >> 1][s][k].y = v.x;
      y[e >> 1][s][k].y = v.y;
    } else {
      x[e >> 1][s][k].x = v.x;
      y[e >> 1][s][k].x = v.y;
    }
  }
};

// f(integral_constant<0>) .. f(integral_constant<K - 1>), unrolled
template <int K, typename F>
__device__ __forceinline__ void pair_unroll(F&& f) {
  if constexpr (K > 0) {
    pair_unroll<K - 1>(f);
    f(std::integral_constant<int, K - 1>());
  }
}

// Non-blocking test of the phase of parity `par`.
__device__ __forceinline__ bool mbar_ready(uint32_t mbar, uint32_t par) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(par)
      : "memory");
  return ok != 0;
}
// Blocking wait (try_wait, system-dependent suspension) for the phase of
// parity `par`; false once *abort is set (by this or another thread) or after
// tc::kWaitCycles, which sets it.
__device__ __noinline__ bool pair_wait_slow(uint32_t mbar, uint32_t par, volatile int* abort) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(par)
        : "memory");
    if (ok) return true;
    if (*abort) return false;
    if (clock64() - t0 > tc::kWaitCycles) {
      *abort = 1;
      return false;
    }
  }
}
__device__ __forceinline__ bool pair_wait(uint32_t mbar, uint32_t par, volatile int* abort) {
  return mbar_ready(mbar, par) || pair_wait_slow(mbar, par, abort);
}
// The stage's full barrier receives one arrival once every cp.async this
// thread issued before has completed (the arrival counts against the
// barrier's expected count).
__device__ __forceinline__ void cp_async_arrive(uint32_t mbar) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(mbar) : "memory");
}

// MINB: CTAs per SM the register allocation must allow (2 caps a one-tile
// CTA at 128 registers per thread; 1 lets N <= 5 keep every accumulator and
// address in registers)
template <int N, int NSLOT, bool SYN, int HALVES, int MINB = 1>
__global__ void __launch_bounds__(256 * HALVES, MINB)
k_contract_pair(const ContractDesc<float>* __restrict__ descs, const PairTask* __restrict__ tasks, CallPtrs ptrs) {
  using G = PairGeom<N, NSLOT, SYN, HALVES>;
  using T = float;
  constexpr int NH = G::NH, ZH = N & 1, NP = N / 2;
  constexpr int STAGES = G::STAGES, KL = G::KL;
  static_assert(KL <= kPairKLMax, "tables are padded for kPairKLMax l per stage");
  static_assert(KL % 2 == 0, "the l parity (accumulator bank) is the position's parity in a stage");
  extern __shared__ __align__(128) unsigned char pair_smem[];
  float* ring = reinterpret_cast<float*>(pair_smem);
  float2* red = reinterpret_cast<float2*>(pair_smem + STAGES * G::BYTES);  // [2][LCH][HALVES][RED_SLAB]
  __shared__ __align__(8) uint64_t full[STAGES], empty[STAGES];
  __shared__ cx<T> cgk[N][N];
  __shared__ int s_abort;

  const PairTask tk = tasks[blockIdx.x];
  const ContractDesc<T>* __restrict__ D = descs + tk.prob;
  const int tid = threadIdx.x;
  const int hh = HALVES == 2 ? (tid >> 8) : 0;          // shared-memory half of this thread
  const bool is_b = HALVES == 2 ? (hh == 1) : (tk.half == 1);
  const bool diag = tk.p == tk.q;
  const bool idle = HALVES == 2 && is_b && diag;        // a diagonal block has one tile
  const int t = tid & 255, w = t >> 5, lane = t & 31;
  const int rg = w;                                     // row group: rows 4 rg .. 4 rg + 3
  const int c = lane;                                   // column
  const int rb = is_b ? tk.q : tk.p, cb = is_b ? tk.p : tk.q;
  const int mpb = 32 * rb + 4 * rg;                     // first row m' (even)
  const int m = 32 * cb + c;
  const bool flip = is_b && !diag;                      // tile B: (-1)^{m'-m} = (-1)^{e+c}
  const int l_start = tk.lstart, l_end = tk.lend;
  const int nst = (l_end - l_start + KL) / KL;          // stages

  if (tid < N * N) {
    const int k = tid / N, g = tid % N;
    const int n = -(N - 1) + 2 * k;
    double sn, cs;
    sincospi((double)(n * g) / (double)N, &sn, &cs);
    cx<T> v;
    if (!SYN) {
      v = mkc<T>((T)cs, (T)sn);  // conj(eta) i^{n} e^{i n gamma_g}
      v = cmul_ipow<T>(v, ((n % 4) + 4) & 3);
      if (D->eta_odd) v = cmul_ipow<T>(v, 3);
    } else {
      const double sc = 2.0 * 3.14159265358979323846 / N;  // eta (2 pi / N) i^{-n} e^{-i n gamma_g}
      v = mkc<T>((T)(cs * sc), (T)(-sn * sc));
      v = cmul_ipow<T>(v, (((-n) % 4) + 4) & 3);
      if (D->eta_odd) v = cmul_ipow<T>(v, 1);
    }
    cgk[k][g] = v;
  }
  const uint32_t ring_s = tc::smem_u32(ring);
  if (tid == 0) {
    s_abort = 0;
    for (int s = 0; s < STAGES; ++s) {
      tc::mbar_init(tc::smem_u32(&full[s]), 256 * HALVES);
      tc::mbar_init(tc::smem_u32(&empty[s]), HALVES * 8);
    }
  }
  __syncthreads();
  volatile int* abort = &s_abort;

  // ---- producer: every thread copies fixed 16-byte chunks of each stage ----
  // The Delta blocks of a stage (16-byte chunk k is Delta floats 4k..) are
  // chunks tid + u NTH, u < DPT, of thread tid: one source pointer and one
  // destination, the others at fixed offsets.  The R rows of each half and
  // (analysis) the f values of each half follow as chunks tid + u NTH of
  // their own numbering.  Source pointers advance by one stage per issue.
  constexpr int NTH = 256 * HALVES;
  constexpr int NCH_D = KL * 256;              // 16-byte chunks of Delta per stage
  static_assert(NCH_D % NTH == 0, "whole Delta chunks per thread");
  constexpr int DPT = NCH_D / NTH;
  constexpr int NCH_R = HALVES * G::R_F / 4;   // of R rows
  constexpr int NCH_F = HALVES * G::F_F / 4;   // of f values
  constexpr int NRF = NCH_R + NCH_F;
  constexpr int CPT = (NRF + NTH - 1) / NTH;
  const float* dsrc = D->dpair + tk.dbase + (size_t)tid * 4;
  const uint32_t ddst = (uint32_t)((tid >> 8) * G::DL + ((tid >> 3) & 31) * G::DP + (tid & 7) * 4) * 4;
  const float* csrc[CPT];
  int cadv[CPT];
  uint32_t cdst[CPT];
  bool cok[CPT];
#pragma unroll
  for (int u = 0; u < CPT; ++u) {
    const int ch = tid + u * NTH;
    cok[u] = ch < NRF;
    csrc[u] = D->dpair;
    cadv[u] = 0;
    cdst[u] = 0;
    if (!cok[u]) continue;
    if (ch < NCH_R) {
      const int fo = ch * 4, h = fo / G::R_F, o = fo % G::R_F;
      const bool hb = HALVES == 2 ? (h == 1) : is_b;
      csrc[u] = D->RSp + ((size_t)(hb ? tk.q : tk.p) * D->Lr + l_start) * G::RROW + o;
      cdst[u] = (uint32_t)(G::R_OFF + fo) * 4;
      cadv[u] = KL * G::RROW;
    } else {
      constexpr int FF = G::F_F > 0 ? G::F_F : 1;
      const int fo = (ch - NCH_R) * 4, h = fo / FF, o = fo % FF;
      const bool hb = HALVES == 2 ? (h == 1) : is_b;
      csrc[u] = reinterpret_cast<const float*>(D->fP + ((size_t)(hb ? tk.p : tk.q) * D->Lrf + l_start) * 32) + o;
      cdst[u] = (uint32_t)(G::F_OFF + fo) * 4;
      cadv[u] = KL * 64;
    }
  }
  const uint32_t full_s = tc::smem_u32(&full[0]), empty_s = tc::smem_u32(&empty[0]);
  auto issue = [&](uint32_t slot) {  // stages in order, each into its slot
    const uint32_t so = ring_s + slot * (uint32_t)G::BYTES;
#pragma unroll
    for (int u = 0; u < DPT; ++u)
      cp_async16_s(so + ddst + (uint32_t)(u * (NTH / 256) * G::DL * 4), dsrc + u * NTH * 4);
    dsrc += KL * 1024;
#pragma unroll
    for (int u = 0; u < CPT; ++u) {
      if (cok[u]) cp_async16_s(so + cdst[u], csrc[u]);
      csrc[u] += cadv[u];
    }
    cp_async_arrive(full_s + 8u * slot);
  };
  {
    const int npre = nst < STAGES ? nst : STAGES;
    for (int i = 0; i < npre; ++i) issue((uint32_t)i);
  }

  constexpr bool BUILTIN = HALVES == 2;  // packed FP32 builtins, else inline PTX
  using AccT = std::conditional_t<BUILTIN, AccF2<4, NSLOT, N>, Acc<T, 4, NSLOT, N, true>>;
  AccT acc;
#pragma unroll
  for (int e = 0; e < 4; ++e)
#pragma unroll
    for (int s = 0; s < NSLOT; ++s)
#pragma unroll
      for (int k = 0; k < N; ++k) acc.set(e, s, k, mkc<T>(0, 0));

  int cur[2] = {-1, -1};
  int sidx = 0;
  int next_b = l_start;  // first l of the next l-segment (scale change in a slot)
  int rbuf = 0;

  // analysis epilogue (gamma step) for slot s holding scale j
  auto flush = [&](int s, int j) {
    const int Lj = D->Lj[j];
    cx<T>* __restrict__ Y = D->Y[j];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int mp = mpb + e;
      if (mp < Lj && m < Lj) {
        cx<T> gk[N];
        if (ZH) gk[N / 2] = acc.get(e, s, 2 * NP);
        const T sgn = ((l_start + e) & 1) ? T(-1) : T(1);
#pragma unroll
        for (int p = 0; p < NP; ++p) {
          const cx<T> b0 = acc.get(e, s, p), b1 = acc.get(e, s, NP + p);
          gk[(N + 1) / 2 + p] = cadd<T>(b0, b1);
          const cx<T> d = csub<T>(b0, b1);
          gk[N / 2 - 1 - p] = mkc<T>(sgn * d.x, sgn * d.y);
        }
        const T fs = (flip && ((e + c) & 1)) ? T(-1) : T(1);
#pragma unroll
        for (int g = 0; g < N; ++g) {
          cx<T> v = mkc<T>(0, 0);
#pragma unroll
          for (int k = 0; k < N; ++k) v = cadd<T>(v, cmul<T>(gk[k], cgk[k][g]));
          Y[((size_t)g * Lj + m) * Lj + mp] = cscale<T>(cmul_ipow<T>(v, (-m) & 3), fs);
        }
      }
    }
  };
  // synthesis prologue (gamma adjoint) for slot s, scale j (or clear)
  auto load = [&](int s, int j) {
    const int Lj = j >= 0 ? D->Lj[j] : 0;
    const cx<T>* __restrict__ V = j >= 0 ? D->Y[j] : nullptr;
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int mp = mpb + e;
      cx<T> h[N];
#pragma unroll
      for (int k = 0; k < N; ++k) h[k] = mkc<T>(0, 0);
      if (mp < Lj && m < Lj) {
#pragma unroll
        for (int g = 0; g < N; ++g) {
          const cx<T> vg = V[((size_t)g * Lj + mp) * Lj + m];
#pragma unroll
          for (int k = 0; k < N; ++k) h[k] = cadd<T>(h[k], cmul<T>(vg, cgk[k][g]));
        }
        const T fs = (flip && ((e + c) & 1)) ? T(-1) : T(1);
#pragma unroll
        for (int k = 0; k < N; ++k) h[k] = cscale<T>(cmul_ipow<T>(h[k], m & 3), fs);
      }
      const T sgn = ((l_start + e) & 1) ? T(-1) : T(1);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const cx<T> hp = h[(N + 1) / 2 + p], hm = h[N / 2 - 1 - p];
        const cx<T> tt = mkc<T>(sgn * hm.x, sgn * hm.y);
        acc.set(e, s, p, cadd<T>(hp, tt));
        acc.set(e, s, NP + p, csub<T>(hp, tt));
      }
      if (ZH) acc.set(e, s, 2 * NP, h[N / 2]);
    }
  };
  // sum of the 8 row groups of each column for `count` l of buffer `buf`
  // (with two halves, each half sums its own tile's partials)
  auto reduce_chunk = [&](int buf, int lfirst, int count) {
    constexpr int SH = HALVES == 2 ? 6 : 5;
    const int lc2 = HALVES == 2 ? ((tid >> 5) & 7) : (tid >> SH), h2 = HALVES == 2 ? (tid >> 8) : 0, c2 = tid & 31;
    if (lc2 < count) {
      const bool b2 = HALVES == 2 ? (h2 == 1) : is_b;
      if (HALVES == 2 && b2 && diag) return;
      const float2* rbp = red + (((size_t)buf * LCH + lc2) * HALVES + h2) * G::RED_SLAB;
      cx<T> sum = mkc<T>(0, 0);
#pragma unroll
      for (int r2 = 0; r2 < 8; ++r2) sum = cadd<T>(sum, rbp[r2 * 32 + c2]);
      const int rb2 = b2 ? tk.q : tk.p, cb2 = b2 ? tk.p : tk.q;
      D->P[((size_t)rb2 * D->L + lfirst + lc2) * D->Lp32 + 32 * cb2 + c2] = sum;
    }
  };

  // slots change scale at l (the start of a new l-segment)
  auto enter = [&](int l) {
    while (D->seg[sidx].hi < l) ++sidx;
    next_b = D->seg[sidx].hi + 1;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      const int jn = D->seg[sidx].j[s];
      if (jn != cur[s]) {
        if (!SYN) {
          if (cur[s] >= 0 && !idle) flush(s, cur[s]);
#pragma unroll
          for (int e = 0; e < 4; ++e)
#pragma unroll
            for (int k = 0; k < N; ++k) acc.set(e, s, k, mkc<T>(0, 0));
        } else if (!idle) {
          load(s, jn);
        }
        cur[s] = jn;
      }
    }
  };

  // the arithmetic of one l (no checks); bank = parity of l - l_start
  auto compute = [&](const int l, const float* S, auto bank) {
    constexpr int BQ = (decltype(bank)::value & 1) * NP;
    constexpr int DB = decltype(bank)::value * G::DL;
    float dv[4];
    if (!is_b) {
#pragma unroll
      for (int e = 0; e < 4; ++e) dv[e] = S[DB + (4 * rg + e) * G::DP + c];
    } else {
      const float4 v = *reinterpret_cast<const float4*>(S + DB + c * G::DP + 4 * rg);
      dv[0] = v.x;
      dv[1] = v.y;
      dv[2] = v.z;
      dv[3] = v.w;
    }
    const float* Rr = S + G::R_OFF + hh * G::R_F + decltype(bank)::value * G::RROW + 4 * rg;
    if (!SYN) {
      const float2 fv = reinterpret_cast<const float2*>(S + G::F_OFF + hh * G::F_F + decltype(bank)::value * 64)[c];
      if constexpr (BUILTIN) {
        const float2 fx = make_float2(fv.x, fv.x), fy = make_float2(fv.y, fv.y);
        const float2 d01 = make_float2(dv[0], dv[1]), d23 = make_float2(dv[2], dv[3]);
        const float2 tx0 = __fmul2_rn(d01, fx), tx1 = __fmul2_rn(d23, fx), ty0 = __fmul2_rn(d01, fy),
                     ty1 = __fmul2_rn(d23, fy);
#pragma unroll
        for (int s = 0; s < NSLOT; ++s)
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
            const float4 r4 = *reinterpret_cast<const float4*>(Rr + (s * NH + h) * 32);
            const float2 rx = make_float2(r4.x, r4.y), ry = make_float2(r4.z, r4.w);
            acc.x[0][s][q] = __ffma2_rn(tx0, rx, acc.x[0][s][q]);
            acc.y[0][s][q] = __ffma2_rn(ty0, rx, acc.y[0][s][q]);
            acc.x[1][s][q] = __ffma2_rn(tx1, ry, acc.x[1][s][q]);
            acc.y[1][s][q] = __ffma2_rn(ty1, ry, acc.y[1][s][q]);
          }
      } else {
        const f2p fx = pk2(fv.x, fv.x), fy = pk2(fv.y, fv.y);
        const f2p d01 = pk2(dv[0], dv[1]), d23 = pk2(dv[2], dv[3]);
        const f2p tx0 = mul2(d01, fx), tx1 = mul2(d23, fx), ty0 = mul2(d01, fy), ty1 = mul2(d23, fy);
#pragma unroll
        for (int s = 0; s < NSLOT; ++s)
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
            const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(Rr + (s * NH + h) * 32);
            acc.x[0][s][q] = fma2(tx0, r.x, acc.x[0][s][q]);
            acc.y[0][s][q] = fma2(ty0, r.x, acc.y[0][s][q]);
            acc.x[1][s][q] = fma2(tx1, r.y, acc.x[1][s][q]);
            acc.y[1][s][q] = fma2(ty1, r.y, acc.y[1][s][q]);
          }
      }
    } else {
      cx<T> part;
      if constexpr (BUILTIN) {
        float2 px0 = make_float2(0.f, 0.f), py0 = px0, px1 = px0, py1 = px0;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s)
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
            const float4 r4 = *reinterpret_cast<const float4*>(Rr + (s * NH + h) * 32);
            const float2 rx = make_float2(r4.x, r4.y), ry = make_float2(r4.z, r4.w);
            px0 = __ffma2_rn(acc.x[0][s][q], rx, px0);
            py0 = __ffma2_rn(acc.y[0][s][q], rx, py0);
            px1 = __ffma2_rn(acc.x[1][s][q], ry, px1);
            py1 = __ffma2_rn(acc.y[1][s][q], ry, py1);
          }
        const float2 d01 = make_float2(dv[0], dv[1]), d23 = make_float2(dv[2], dv[3]);
        const float2 sx = __ffma2_rn(d23, px1, __fmul2_rn(d01, px0)), sy = __ffma2_rn(d23, py1, __fmul2_rn(d01, py0));
        part.x = sx.x + sx.y;
        part.y = sy.x + sy.y;
      } else {
        f2p px0 = 0, py0 = 0, px1 = 0, py1 = 0;
#pragma unroll
        for (int s = 0; s < NSLOT; ++s)
#pragma unroll
          for (int h = 0; h < NH; ++h) {
            const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
            const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(Rr + (s * NH + h) * 32);
            px0 = fma2(acc.x[0][s][q], r.x, px0);
            py0 = fma2(acc.y[0][s][q], r.x, py0);
            px1 = fma2(acc.x[1][s][q], r.y, px1);
            py1 = fma2(acc.y[1][s][q], r.y, py1);
          }
        const f2p d01 = pk2(dv[0], dv[1]), d23 = pk2(dv[2], dv[3]);
        const f2p sx = fma2(d23, px1, mul2(d01, px0)), sy = fma2(d23, py1, mul2(d01, py0));
        float a, b2;
        upk2(sx, a, b2);
        part.x = a + b2;
        upk2(sy, a, b2);
        part.y = a + b2;
      }
      const int lc = (l - l_start) & (LCH - 1);
      red[(((size_t)rbuf * LCH + lc) * HALVES + hh) * G::RED_SLAB + rg * 32 + c] = part;
    }
  };

  static_assert((LCH & (LCH - 1)) == 0 && LCH % KL == 0, "l-chunks of whole stages");
  enter(l_start);
  for (int i = 0; i < nst; ++i) {
    const int l0 = l_start + KL * i;
    if (SYN && i > 0 && ((KL * i) & (LCH - 1)) == 0) {
      // the chunk's partials are in red: with two halves, each half waits
      // for its own warps only (named barrier 1 + half, 256 threads)
      if (HALVES == 2) asm volatile("bar.sync %0, 256;" ::"r"(1 + hh) : "memory");
      else __syncthreads();
      rbuf ^= 1;
      reduce_chunk(rbuf ^ 1, l0 - LCH, LCH);
    }
    // ring slot and phase parity of stage i (shifts for a power-of-two depth)
    const uint32_t slot = (uint32_t)i % STAGES, par = ((uint32_t)i / STAGES) & 1u;
    if (pair_wait(full_s + 8u * slot, par, abort)) {
      const float* S = ring + slot * G::SIZE;
      if (l0 + KL - 1 < next_b && l0 + KL - 1 <= l_end) {  // every l inside the current segment
        if (!idle) pair_unroll<KL>([&](auto kk) { compute(l0 + decltype(kk)::value, S, kk); });
      } else {
#pragma unroll 1
        for (int kk = 0; kk < KL; ++kk) {
          const int l = l0 + kk;
          if (l > l_end) break;
          if (l >= next_b) enter(l);
          if (idle) continue;
          pair_unroll<KL>([&](auto kc) {
            if (kk == decltype(kc)::value) compute(l, S, kc);
          });
        }
      }
    }
    __syncwarp();
    if (lane == 0) tc::mbar_arrive(empty_s + 8u * slot);
    // refill the slot read LAG stages ago (every warp has normally left it)
    // with stage r + STAGES; after a timeout the wait returns false at once
    const int r = i - G::LAG;
    if (r >= 0 && r + STAGES < nst) {
      const uint32_t rslot = (uint32_t)r % STAGES, rpar = ((uint32_t)r / STAGES) & 1u;
      if (pair_wait(empty_s + 8u * rslot, rpar, abort)) issue(rslot);
    }
  }
  cp_async_wait<0>();  // this thread's copies (all consumed, unless a wait gave up)
  if (SYN) {
    __syncthreads();
    const int n_it = l_end - l_start + 1;
    const int last = (n_it - 1) % LCH + 1;  // entries in the final chunk
    const int lfirst = l_end - last + 1;
    // the final chunk sits in rbuf unless it was full and already swapped
    reduce_chunk(rbuf, lfirst, last);
  } else if (!idle) {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s)
      if (cur[s] >= 0) flush(s, cur[s]);
  }
  if (*abort && tid == 0) atomicAdd(&g_pair_timeouts, 1);
}

}  // namespace s2dw
