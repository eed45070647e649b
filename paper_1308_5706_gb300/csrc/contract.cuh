// Fused l-contraction kernels (Sec. 3.2 Eq. (27); Sec. 3.3 Eqs. (34) and (32)).
//
// Analysis: for each (m', m) with m', m >= 0 and each scale j,
//   G^j_{m'mk} = sum_{l in supp kappa^j} Delta^l_{m'm} f_lm R^j_{l m' k},
//   R^j_{l m' k} = Delta^l_{m' n_k} kappa^j(l) |s_{l n_k}|,
// followed by the gamma step (Eq. (28)) as an epilogue:
//   Y^j_g[m][m'] = i^{-m} sum_k G^j_{m'mk} conj(eta) i^{n_k} e^{i n_k gamma_g}
// (stored with m' fastest, so the beta step reads contiguous columns; the
// synthesis input Vhat_g[m'][m] is stored with m fastest, so this prologue
// reads it coalesced).
// Since Psi^j*_ln = kappa^j(l) conj(eta) |s_ln|, conj(eta) i^{n-m} G is the
// cube U_{m m' n} of Eq. (27) for m' >= 0 (U_{m,-m',n} = (-1)^{m+n} U_{m m' n}).
//
// Synthesis (adjoint): the tile holds, for each (m', m) and scale j,
//   H^j_{m'mk} = eta i^{m-n_k} (2 pi/N) sum_g Vhat^j_g[m'][m] e^{-i n_k gamma_g}
// (gamma quadrature of Eq. (39) with z_n = 1/N), and produces for every l
//   partial_l(m) = sum_{m' in tile} Delta^l_{m'm} sum_{j,k} R^j_{l m' k} H^j_{m'mk},
// reduced over the tile's m' rows in shared memory; a second kernel sums the
// tiles in a fixed order (deterministic, no atomics) and applies (2l+1)/(8 pi^2).
//
// Each l has at most two active scales (the open supports of kappa^j and
// kappa^{j-2} are disjoint), held in two accumulator slots (j % 2).
//
// Data movement: per l, the tile's Delta block (stored rows m' x columns m,
// and for tiles below the diagonal the stored rows m x columns m'), the 32
// values f_lm and the R rows are copied by cp.async into a ring of S stages
// (up to 8, as two CTAs per SM allow) in shared memory, issued S-2 stages
// ahead; one barrier per two l (the barrier round trip, not arithmetic,
// bounded a loop with one barrier per l).
// Thread layout: 256 threads, each owning E consecutive rows m' and one
// column m of a (8E x 32) tile.  Tiles with every row above every column map
// lanes along m' so that their reads of the transposed block stay conflict free.
#pragma once

#include <type_traits>

#include "internal.h"

namespace s2dw {

constexpr int kMaxStages = 8;
constexpr size_t kCtaSmemBudget = 112 * 1024;  // two CTAs per SM (228 KB, 1 KB reserved each)


// E consecutive values from 16-byte aligned shared memory.
template <typename T, int E> struct VecLdS;
template <> struct VecLdS<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&r)[4]) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
};
template <> struct VecLdS<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&r)[2]) {
    const double2 v = *reinterpret_cast<const double2*>(p);
    r[0] = v.x; r[1] = v.y;
  }
};

// Accumulators of a thread: E elements x NSLOT slots x N orders, complex.
// Generic form: cx<T> per entry.  float with E = 4: real and imaginary parts
// of element pairs (0,1), (2,3) packed for f32x2 instructions.
template <typename T, int E, int NSLOT, int N, bool PACK> struct Acc;
template <typename T, int E, int NSLOT, int N> struct Acc<T, E, NSLOT, N, false> {
  cx<T> v[E][NSLOT][N];
  __device__ __forceinline__ cx<T> get(int e, int s, int k) const { return v[e][s][k]; }
  __device__ __forceinline__ void set(int e, int s, int k, cx<T> x) { v[e][s][k] = x; }
};
template <int E, int NSLOT, int N> struct Acc<float, E, NSLOT, N, true> {
  f2p x[E / 2][NSLOT][N], y[E / 2][NSLOT][N];
  __device__ __forceinline__ cx<float> get(int e, int s, int k) const {
    float a0, a1, b0, b1;
    upk2(x[e >> 1][s][k], a0, a1);
    upk2(y[e >> 1][s][k], b0, b1);
    return (e & 1) ? mkc<float>(a1, b1) : mkc<float>(a0, b0);
  }
  __device__ __forceinline__ void set(int e, int s, int k, cx<float> v) {
    float a0, a1, b0, b1;
    upk2(x[e >> 1][s][k], a0, a1);
    upk2(y[e >> 1][s][k], b0, b1);
    if (e & 1) {
      a1 = v.x;
      b1 = v.y;
    } else {
      a0 = v.x;
      b0 = v.y;
    }
    x[e >> 1][s][k] = pk2(a0, a1);
    y[e >> 1][s][k] = pk2(b0, b1);
  }
};

// Shared-memory geometry of one pipeline stage (element counts of T).
template <typename T, int N, int NSLOT, int E>
struct StageGeom {
  static constexpr int TMP = 8 * E;                 // tile rows (m')
  static constexpr int EPC = 16 / sizeof(T);        // elements per 16-byte chunk
  static constexpr int APITCH = TILE + EPC;         // block A: [TMP][APITCH], stored rows m' x cols m
  static constexpr int BPITCH = TMP;                // block B: [TILE][BPITCH], stored rows m x cols m'
  static constexpr int A_OFF = 0;
  static constexpr int B_OFF = A_OFF + TMP * APITCH;
  static constexpr int F_OFF = B_OFF + TILE * BPITCH;         // TILE complex = 2*TILE elements
  static constexpr int R_OFF = F_OFF + 2 * TILE;              // [NSLOT][(N+1)/2][TMP], n_k >= 0
  static constexpr int SIZE = R_OFF + NSLOT * ((N + 1) / 2) * TMP;
  static constexpr size_t BYTES = (size_t)SIZE * sizeof(T);
};

template <typename T, bool SYN>
__host__ __device__ constexpr size_t contract_red_bytes() {
  return SYN ? 2 * LCH * 8 * TILE * sizeof(cx<T>) : 0;
}
// ring depth: as many stages as fit next to the reduction buffer (4..8, even)
template <typename T, int N, int NSLOT, bool SYN, int E>
__host__ __device__ constexpr int contract_stages() {
  const size_t fit = (kCtaSmemBudget - contract_red_bytes<T, SYN>()) / StageGeom<T, N, NSLOT, E>::BYTES;
  const int s = fit > (size_t)kMaxStages ? kMaxStages : (fit < 4 ? 4 : (int)fit);
  return s & ~1;
}
template <typename T, int N, int NSLOT, bool SYN, int E>
__host__ __device__ constexpr size_t contract_smem_bytes() {
  return contract_stages<T, N, NSLOT, SYN, E>() * StageGeom<T, N, NSLOT, E>::BYTES + contract_red_bytes<T, SYN>();
}

// Two CTAs per SM (128 registers) where the accumulators allow it (FP32, N <= 5).
template <typename T, int N, int NSLOT, bool SYN, int E>
__global__ void __launch_bounds__(256, (sizeof(T) == 4 && N <= 5 ? 2 : 1))
k_contract(const ContractDesc<T>* __restrict__ descs, const TileTask* __restrict__ tiles, CallPtrs ptrs) {
  using G = StageGeom<T, N, NSLOT, E>;
  constexpr int STAGES = contract_stages<T, N, NSLOT, SYN, E>();
  // Order parity: R_{l m' -n} = (-1)^{l+m'} R_{l m' n}, so only n >= 0 is
  // staged (NH rows, row 0 is n = 0 when N is odd) and the sums over l of a
  // pair +-n run as two banks, l of the parity of l_start (bank 0) and the
  // other (bank 1): analysis G_{+n} = B0 + B1 and G_{-n} = (-1)^{m'+l_start}
  // (B0 - B1); synthesis folds H_{+n} +- (-1)^{m'+l_start} H_{-n} into the
  // bank of each parity.  Accumulator index q: bank 0 orders n > 0 in
  // [0, NP), bank 1 in [NP, 2 NP), n = 0 at 2 NP.  Rows m' of a thread start
  // at an even m', so (-1)^{m'} = (-1)^e.
  constexpr int NH = (N + 1) / 2, ZH = N & 1, NP = N / 2;
  static_assert(E % 2 == 0, "row parity of element e must be (-1)^e");
  constexpr int RG = 8;
  constexpr int TMP = G::TMP;
  constexpr int EPC = G::EPC;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* ring = reinterpret_cast<T*>(smem_raw);
  cx<T>* red = reinterpret_cast<cx<T>*>(smem_raw + STAGES * G::BYTES);  // [2][LCH][RG][TILE]
  __shared__ cx<T> cgk[N][N];

  const TileTask tk = tiles[blockIdx.x];
  const ContractDesc<T>* __restrict__ D = descs + tk.prob;
  const int Lp = D->Lp;
  const T* __restrict__ delta = D->delta;
  const T* __restrict__ RS = D->RS;
  const int mp0 = tk.bmp * TMP, m0 = tk.bm * TILE;
  const bool ttile = mp0 > m0 + TILE - 1;                 // every row above every column
  const bool need_a = m0 + TILE - 1 >= (mp0 & ~3);        // some entry stored as (m', m)
  const bool need_b = m0 < ((mp0 + TMP - 1) & ~3);        // some entry stored as (m, m')
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int c, rg;
  if (!ttile) {
    rg = w;
    c = lane;
  } else {
    c = (w << 2) + (lane >> 3);
    rg = lane & 7;
  }
  const int m = m0 + c;
  const int mpb = mp0 + E * rg;
  const bool tr = m < (mpb & ~3);
  const T sg0 = ((mpb - m) & 1) ? T(-1) : T(1);

  if (threadIdx.x < N * N) {
    const int k = threadIdx.x / N, g = threadIdx.x % N;
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

  const cx<T>* __restrict__ f = SYN ? nullptr : reinterpret_cast<const cx<T>*>(ptrs.f[tk.prob]);
  const int l_start = tk.lstart, l_end = tk.lend;

  // ---- producer: stage the operands of iteration l into ring slot st ----
  // Per-thread copy roles are fixed for the whole tile; only the slab, f and
  // R offsets move with l, and they advance incrementally (issue() is called
  // for l_start, l_start+1, ... in order).  Offsets are 32-bit element
  // offsets (a table of L = 2048 has 1.44e9 entries) and destinations 32-bit
  // shared addresses.  Rows of the Delta block past the slab (m' or m > l)
  // are copied unguarded: they read neighbouring table entries (finite; the
  // table has a zero front pad for the rows of small l that start before it)
  // and meet zero R rows (m' > l) or zero f (m > l).
  const int t = threadIdx.x;
  constexpr int CPRA = TILE / EPC, CPRB = TMP / EPC, CPRR = TMP / EPC;
  constexpr int FCH = 2 * TILE / EPC, CPC = EPC / 2, NRCH = NSLOT * NH * CPRR;
  const bool do_a = need_a && t < TMP * CPRA;
  const bool do_b = need_b && t < TILE * CPRB;
  const int ra = mp0 + t / CPRA, rb = m0 + t / CPRB;
  const int a_A = delta_row_A(ra, m0 + (t % CPRA) * EPC), a_B = delta_row_B(ra);
  const int b_A = delta_row_A(rb, mp0 + (t % CPRB) * EPC), b_B = delta_row_B(rb);
  const uint32_t ring_s = (uint32_t)__cvta_generic_to_shared(ring);
  const uint32_t a_dst = ring_s + (uint32_t)(G::A_OFF + (t / CPRA) * G::APITCH + (t % CPRA) * EPC) * sizeof(T);
  const uint32_t b_dst = ring_s + (uint32_t)(G::B_OFF + (t / CPRB) * G::BPITCH + (t % CPRB) * EPC) * sizeof(T);
  const int fq = t - 256 + FCH;
  const int f_mm = m0 + fq * CPC;
  const uint32_t f_dst = ring_s + (uint32_t)(G::F_OFF + fq * EPC) * sizeof(T);
  const bool do_r = t < NRCH;
  const uint32_t r_dst = ring_s + (uint32_t)(G::R_OFF + (t / CPRR) * TMP + (t % CPRR) * EPC) * sizeof(T);
  int is_slab = (int)delta_slab_offset(l_start);  // state of the next issue
  int is_f = l_start * l_start + l_start + f_mm;
  int is_rs = l_start * (NSLOT * NH) * Lp + (t / CPRR) * Lp + mp0 + (t % CPRR) * EPC;
  int is_l = l_start;
  int wr = 0;  // ring slot of the next issue
  auto issue = [&]() {
    const int l = is_l;
    if (l <= l_end) {
      const uint32_t so = (uint32_t)wr * (uint32_t)G::BYTES;
      const int cl = (l >> 2) + 1;
      if (do_a) cp_async16_s(a_dst + so, delta + (is_slab + a_A + a_B * cl));
      if (do_b) cp_async16_s(b_dst + so, delta + (is_slab + b_A + b_B * cl));
      if (!SYN && fq >= 0) {
        // f_lm for m in [m0, m0 + TILE), zero beyond m = l (the array ends at l = L-1)
        const int nvalid = min(CPC, max(0, l + 1 - f_mm));
        cp_async16_s(f_dst + so, f + (nvalid > 0 ? is_f : 0), nvalid * (int)sizeof(cx<T>));
      }
      if (do_r) cp_async16_s(r_dst + so, RS + is_rs);
      is_slab += 8 * cl * (cl + 1);
      is_f += 2 * (l + 1);
      is_rs += (NSLOT * NH) * Lp;
      is_l = l + 1;
    }
    wr = (wr + 1 == STAGES) ? 0 : wr + 1;
    cp_async_commit();
  };

#pragma unroll
  for (int i = 0; i < STAGES - 2; ++i) issue();

  constexpr bool PACK = std::is_same<T, float>::value && E == 4;
  Acc<T, E, NSLOT, N, PACK> acc;
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int s = 0; s < NSLOT; ++s)
#pragma unroll
      for (int k = 0; k < N; ++k) acc.set(e, s, k, mkc<T>(0, 0));

  int cur[2] = {-1, -1};
  int sidx = 0;
  while (sidx < D->nseg && D->seg[sidx].hi < l_start) ++sidx;
  int seg_hi = -1;
  int rbuf = 0;

  // analysis epilogue (gamma step) for slot s holding scale j
  auto flush = [&](int s, int j) {
    const int Lj = D->Lj[j];
    cx<T>* __restrict__ Y = D->Y[j];
#pragma unroll
    for (int e = 0; e < E; ++e) {
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
#pragma unroll
        for (int g = 0; g < N; ++g) {
          cx<T> v = mkc<T>(0, 0);
#pragma unroll
          for (int k = 0; k < N; ++k) v = cadd<T>(v, cmul<T>(gk[k], cgk[k][g]));
          Y[((size_t)g * Lj + m) * Lj + mp] = cmul_ipow<T>(v, (-m) & 3);
        }
      }
    }
  };
  // synthesis prologue (gamma adjoint) for slot s, scale j (or clear)
  auto load = [&](int s, int j) {
    const int Lj = j >= 0 ? D->Lj[j] : 0;
    const cx<T>* __restrict__ V = j >= 0 ? D->Y[j] : nullptr;
#pragma unroll
    for (int e = 0; e < E; ++e) {
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
#pragma unroll
        for (int k = 0; k < N; ++k) h[k] = cmul_ipow<T>(h[k], m & 3);
      }
      const T sgn = ((l_start + e) & 1) ? T(-1) : T(1);
#pragma unroll
      for (int p = 0; p < NP; ++p) {
        const cx<T> hp = h[(N + 1) / 2 + p], hm = h[N / 2 - 1 - p];
        const cx<T> t = mkc<T>(sgn * hm.x, sgn * hm.y);
        acc.set(e, s, p, cadd<T>(hp, t));
        acc.set(e, s, NP + p, csub<T>(hp, t));
      }
      if (ZH) acc.set(e, s, 2 * NP, h[N / 2]);
    }
  };
  auto reduce_chunk = [&](int buf, int lfirst, int count) {
    const int lc2 = threadIdx.x >> 5, c2 = threadIdx.x & 31;
    if (lc2 < count) {
      const cx<T>* rb = red + (size_t)buf * LCH * RG * TILE;
      cx<T> sum = mkc<T>(0, 0);
#pragma unroll
      for (int r2 = 0; r2 < RG; ++r2) sum = cadd<T>(sum, rb[(lc2 * RG + r2) * TILE + c2]);
      D->P[((size_t)tk.bmp * D->L + lfirst + lc2) * D->Lp32 + m0 + c2] = sum;
    }
  };

  __syncthreads();  // cgk visible
  // Two l per barrier: stages it, it+1 are waited for together and stages
  // it+S-2, it+S-1 are issued into the slots that l-2, l-1 have released.
  int rd = 0;  // ring slot of the next iteration processed
  auto process = [&](const int l, const int it, auto bank) {
    constexpr int BQ = decltype(bank)::value * NP;  // first accumulator of this l's bank
    // slot occupancy changes at segment boundaries
    if (l > seg_hi) {
      while (D->seg[sidx].hi < l) ++sidx;
      seg_hi = D->seg[sidx].hi;
#pragma unroll
      for (int s = 0; s < NSLOT; ++s) {
        const int jn = D->seg[sidx].j[s];
        if (jn != cur[s]) {
          if (!SYN) {
            if (cur[s] >= 0) flush(s, cur[s]);
#pragma unroll
            for (int e = 0; e < E; ++e)
#pragma unroll
              for (int k = 0; k < N; ++k) acc.set(e, s, k, mkc<T>(0, 0));
          } else {
            load(s, jn);
          }
          cur[s] = jn;
        }
      }
    }
    const T* S = ring + rd * G::SIZE;
    rd = (rd + 1 == STAGES) ? 0 : rd + 1;
    // Every element computes: out-of-range rows and columns contribute exact
    // zeros (zero R rows for m' > l or inactive slots, zero-filled f for
    // m > l, zero H outside a scale's band), and synthesis partials of
    // columns m > l are never read.
    cx<T> part = mkc<T>(0, 0);
    {
      T dv[E];
      if (!tr) {
#pragma unroll
        for (int e = 0; e < E; ++e) dv[e] = S[G::A_OFF + (mpb - mp0 + e) * G::APITCH + c];
      } else {
        VecLdS<T, E>::ld(S + G::B_OFF + c * G::BPITCH + (mpb - mp0), dv);
#pragma unroll
        for (int e = 0; e < E; ++e) dv[e] *= (e & 1) ? -sg0 : sg0;
      }
      const T* Rr = S + G::R_OFF + (mpb - mp0);
      if constexpr (PACK) {
        // float, E = 4: pairs (0,1) and (2,3) per f32x2 instruction
        if (!SYN) {
          const cx<T> fv = reinterpret_cast<const cx<T>*>(S + G::F_OFF)[c];
          const f2p fx = pk2(fv.x, fv.x), fy = pk2(fv.y, fv.y);
          const f2p d01 = pk2(dv[0], dv[1]), d23 = pk2(dv[2], dv[3]);
          const f2p tx0 = mul2(d01, fx), tx1 = mul2(d23, fx), ty0 = mul2(d01, fy), ty1 = mul2(d23, fy);
#pragma unroll
          for (int s = 0; s < NSLOT; ++s)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
              const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(Rr + (s * NH + h) * TMP);
              acc.x[0][s][q] = fma2(tx0, r.x, acc.x[0][s][q]);
              acc.y[0][s][q] = fma2(ty0, r.x, acc.y[0][s][q]);
              acc.x[1][s][q] = fma2(tx1, r.y, acc.x[1][s][q]);
              acc.y[1][s][q] = fma2(ty1, r.y, acc.y[1][s][q]);
            }
        } else {
          f2p px0 = 0, py0 = 0, px1 = 0, py1 = 0;
#pragma unroll
          for (int s = 0; s < NSLOT; ++s)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
              const ulonglong2 r = *reinterpret_cast<const ulonglong2*>(Rr + (s * NH + h) * TMP);
              px0 = fma2(acc.x[0][s][q], r.x, px0);
              py0 = fma2(acc.y[0][s][q], r.x, py0);
              px1 = fma2(acc.x[1][s][q], r.y, px1);
              py1 = fma2(acc.y[1][s][q], r.y, py1);
            }
          const f2p d01 = pk2(dv[0], dv[1]), d23 = pk2(dv[2], dv[3]);
          const f2p sx = fma2(d23, px1, mul2(d01, px0)), sy = fma2(d23, py1, mul2(d01, py0));
          float a, b;
          upk2(sx, a, b);
          part.x = a + b;
          upk2(sy, a, b);
          part.y = a + b;
        }
      } else {
        if (!SYN) {
          const cx<T> fv = reinterpret_cast<const cx<T>*>(S + G::F_OFF)[c];
          cx<T> tt[E];
#pragma unroll
          for (int e = 0; e < E; ++e) tt[e] = mkc<T>(dv[e] * fv.x, dv[e] * fv.y);
#pragma unroll
          for (int s = 0; s < NSLOT; ++s)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
              T r[E];
              VecLdS<T, E>::ld(Rr + (s * NH + h) * TMP, r);
#pragma unroll
              for (int e = 0; e < E; ++e) {
                cx<T>& a = acc.v[e][s][q];
                a.x = fma(tt[e].x, r[e], a.x);
                a.y = fma(tt[e].y, r[e], a.y);
              }
            }
        } else {
          cx<T> p[E];
#pragma unroll
          for (int e = 0; e < E; ++e) p[e] = mkc<T>(0, 0);
#pragma unroll
          for (int s = 0; s < NSLOT; ++s)
#pragma unroll
            for (int h = 0; h < NH; ++h) {
              const int q = (ZH && h == 0) ? 2 * NP : BQ + h - ZH;
              T r[E];
              VecLdS<T, E>::ld(Rr + (s * NH + h) * TMP, r);
#pragma unroll
              for (int e = 0; e < E; ++e) {
                const cx<T> a = acc.v[e][s][q];
                p[e].x = fma(a.x, r[e], p[e].x);
                p[e].y = fma(a.y, r[e], p[e].y);
              }
            }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            part.x = fma(dv[e], p[e].x, part.x);
            part.y = fma(dv[e], p[e].y, part.y);
          }
        }
      }
    }
    if (SYN) {
      const int lc = it % LCH;
      red[((size_t)rbuf * LCH + lc) * RG * TILE + rg * TILE + c] = part;
      if (lc == LCH - 1) rbuf ^= 1;
    }
  };
  const int n_it = l_end - l_start + 1;
  for (int it = 0; it < n_it; it += 2) {
    cp_async_wait<STAGES - 4>();
    __syncthreads();
    issue();
    issue();
    if (SYN && it > 0 && (it % LCH) == 0) reduce_chunk(rbuf ^ 1, l_start + it - LCH, LCH);
    process(l_start + it, it, std::integral_constant<int, 0>());
    if (it + 1 < n_it) process(l_start + it + 1, it + 1, std::integral_constant<int, 1>());
  }
  cp_async_wait<0>();
  if (SYN) {
    __syncthreads();
    const int n_it = l_end - l_start + 1;
    const int last = (n_it - 1) % LCH + 1;         // entries in the final chunk
    const int lfirst = l_end - last + 1;
    const int buf = (last == LCH) ? (rbuf ^ 1) : rbuf;
    reduce_chunk(buf, lfirst, last);
  } else {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s)
      if (cur[s] >= 0) flush(s, cur[s]);
  }
}

// f_lm = (2l+1)/(8 pi^2) * (sum of tile partials, fixed order), m >= 0, and
// f_{l,-m} = (-1)^m conj(f_lm) (real signal).  blockIdx.z = job.
template <typename T>
__global__ void k_syn_reduce(ReduceJobs jobs, int tmp) {
  const int job = blockIdx.z;
  const int l = blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  const int L = jobs.L[job];
  if (l >= L || m > l) return;
  const ContractDesc<T>* dw = reinterpret_cast<const ContractDesc<T>*>(jobs.dw[job]);
  const ContractDesc<T>* dp = reinterpret_cast<const ContractDesc<T>*>(jobs.dp[job]);
  cx<T> sum = mkc<T>(0, 0);
  if (l <= jobs.lend[job]) {
    const int nb = min(l / tmp, dw->nbr - 1);
    for (int b = 0; b <= nb; ++b) sum = cadd<T>(sum, dw->P[((size_t)b * dw->L + l) * dw->Lp32 + m]);
  }
  if (l < jobs.Lphi[job]) {
    const int nb = min(l / tmp, dp->nbr - 1);
    for (int b = 0; b <= nb; ++b) sum = cadd<T>(sum, dp->P[((size_t)b * dp->L + l) * dp->Lp32 + m]);
  }
  // (2l+1)/(8 pi^2) of the synthesis (Eq. (32)); the forward SHT's plan has
  // Phi_l = sqrt((2l+1)/(4 pi)) and needs f_lm = Phi_l S where the partials
  // carry 2 pi Phi_l S (the N = 1 gamma quadrature), hence 1/(2 pi)
  const T fac = jobs.sht[job] ? (T)(0.5 / 3.14159265358979323846)
                              : (T)((2.0 * l + 1.0) / (8.0 * 3.14159265358979323846 * 3.14159265358979323846));
  sum = cscale<T>(sum, fac);
  cx<T>* __restrict__ out = reinterpret_cast<cx<T>*>(jobs.out[job]);
  out[l * l + l + m] = sum;
  if (m > 0) {
    const cx<T> cj = cconj<T>(sum);
    out[l * l + l - m] = (m & 1) ? mkc<T>(-cj.x, -cj.y) : cj;
  }
}

template <typename T, int N, int NSLOT, bool SYN, int E>
void launch_one(dim3 grid, const ContractDesc<T>* descs, const TileTask* tiles, const CallPtrs& ptrs,
                cudaStream_t st) {
  constexpr size_t smem = contract_smem_bytes<T, N, NSLOT, SYN, E>();
  static unsigned long long dev_done = 0;  // devices on which the smem cap is set
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 64 || !(dev_done & (1ull << dev))) {
    cudaFuncSetAttribute(k_contract<T, N, NSLOT, SYN, E>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev < 64) dev_done |= 1ull << dev;
  }
  k_contract<T, N, NSLOT, SYN, E><<<grid, 256, smem, st>>>(descs, tiles, ptrs);
}

template <typename T, int E>
void launch_contract_impl(int N, int nslot, bool syn, const ContractDesc<T>* descs, const TileTask* tiles,
                          int ntiles, const CallPtrs& ptrs, cudaStream_t st) {
  if (ntiles <= 0) return;
  dim3 grid(ntiles);
#define S2DW_CASE(NN)                                                        \
  case NN:                                                                   \
    if (syn) launch_one<T, NN, 2, true, E>(grid, descs, tiles, ptrs, st);    \
    else launch_one<T, NN, 2, false, E>(grid, descs, tiles, ptrs, st);       \
    break;
  if (N == 1 && nslot == 1) {
    if (syn) launch_one<T, 1, 1, true, E>(grid, descs, tiles, ptrs, st);
    else launch_one<T, 1, 1, false, E>(grid, descs, tiles, ptrs, st);
    return;
  }
  switch (N) {
    S2DW_CASE(1)
    S2DW_CASE(2)
    S2DW_CASE(3)
    S2DW_CASE(4)
    S2DW_CASE(5)
    S2DW_CASE(6)
    S2DW_CASE(7)
    S2DW_CASE(8)
    default: break;
  }
#undef S2DW_CASE
}

}  // namespace s2dw
