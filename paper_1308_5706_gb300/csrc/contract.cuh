// Fused l-contraction kernels (Sec. 3.2 Eq. (27); Sec. 3.3 Eqs. (34) and (32)).
//
// Analysis: for each (m', m) with m', m >= 0 and each scale j,
//   G^j_{m'mk} = sum_{l in supp kappa^j} Delta^l_{m'm} f_lm R^j_{l m' k},
//   R^j_{l m' k} = Delta^l_{m' n_k} kappa^j(l) |s_{l n_k}|,
// followed by the gamma step (Eq. (28)) as an epilogue:
//   Y^j_g[m'][m] = i^{-m} sum_k G^j_{m'mk} conj(eta) i^{n_k} e^{i n_k gamma_g}.
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
// Thread layout: 256 threads, each owning E consecutive rows m' and one
// column m of a (8E x 32) tile.  Tiles with every row above every column
// ("transposed") map lanes along m' so that the Delta loads, which then read
// the stored row m, stay coalesced.
#pragma once

#include "internal.h"

namespace s2dw {

template <typename T, int E> struct VecLd;
template <> struct VecLd<float, 4> {
  static __device__ __forceinline__ void ld(const float* p, float (&r)[4]) {
    float4 v = __ldg(reinterpret_cast<const float4*>(p));
    r[0] = v.x; r[1] = v.y; r[2] = v.z; r[3] = v.w;
  }
};
template <> struct VecLd<double, 2> {
  static __device__ __forceinline__ void ld(const double* p, double (&r)[2]) {
    double2 v = __ldg(reinterpret_cast<const double2*>(p));
    r[0] = v.x; r[1] = v.y;
  }
};
template <> struct VecLd<float, 2> {
  static __device__ __forceinline__ void ld(const float* p, float (&r)[2]) {
    float2 v = __ldg(reinterpret_cast<const float2*>(p));
    r[0] = v.x; r[1] = v.y;
  }
};
template <> struct VecLd<double, 4> {
  static __device__ __forceinline__ void ld(const double* p, double (&r)[4]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p + 2));
    r[0] = a.x; r[1] = a.y; r[2] = b.x; r[3] = b.y;
  }
};

template <typename T> __device__ __forceinline__ cx<T> ldc(const cx<T>* p) { return __ldg(p); }

template <typename T, int N, int NSLOT, bool SYN, int E>
__global__ void __launch_bounds__(256)
k_contract(const ContractDesc<T>* __restrict__ descs, const TileTask* __restrict__ tiles, CallPtrs ptrs) {
  constexpr int RG = 8;            // row groups per tile (= 256 / 32 lanes)
  constexpr int TMP = RG * E;      // tile rows (m')
  __shared__ cx<T> cgk[N][N];
  __shared__ cx<T> red[SYN ? 2 : 1][SYN ? LCH : 1][RG][32];

  const TileTask tk = tiles[blockIdx.x];
  const ContractDesc<T>* __restrict__ D = descs + tk.prob;
  const int Lp = D->Lp;
  const T* __restrict__ delta = D->delta;
  const T* __restrict__ RS = D->RS;
  const int mp0 = tk.bmp * TMP, m0 = tk.bm * TILE;
  const bool ttile = mp0 > m0 + TILE - 1;
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
  int dA[E], dB[E];
  if (!tr) {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      dA[e] = delta_row_A(mpb + e, m);
      dB[e] = delta_row_B(mpb + e);
    }
  } else {
#pragma unroll
    for (int e = 0; e < E; ++e) {
      dA[e] = delta_row_A(m, mpb);
      dB[e] = delta_row_B(m);
    }
  }
  const T sg0 = ((mpb - m) & 1) ? T(-1) : T(1);

  if (threadIdx.x < N * N) {
    const int k = threadIdx.x / N, g = threadIdx.x % N;
    const int n = -(N - 1) + 2 * k;
    double sn, cs;
    sincospi((double)(n * g) / (double)N, &sn, &cs);
    cx<T> v;
    if (!SYN) {
      // conj(eta) i^{n} e^{i n gamma_g}
      v = mkc<T>((T)cs, (T)sn);
      v = cmul_ipow<T>(v, ((n % 4) + 4) & 3);
      if (D->eta_odd) v = cmul_ipow<T>(v, 3);
    } else {
      // eta (2 pi / N) i^{-n} e^{-i n gamma_g}
      const double sc = 2.0 * 3.14159265358979323846 / N;
      v = mkc<T>((T)(cs * sc), (T)(-sn * sc));
      v = cmul_ipow<T>(v, (((-n) % 4) + 4) & 3);
      if (D->eta_odd) v = cmul_ipow<T>(v, 1);
    }
    cgk[k][g] = v;
  }
  __syncthreads();

  cx<T> acc[E][NSLOT][N];
#pragma unroll
  for (int e = 0; e < E; ++e)
#pragma unroll
    for (int s = 0; s < NSLOT; ++s)
#pragma unroll
      for (int k = 0; k < N; ++k) acc[e][s][k] = mkc<T>(0, 0);

  const cx<T>* __restrict__ f = SYN ? nullptr : reinterpret_cast<const cx<T>*>(ptrs.f[tk.prob]);
  const int l_start = tk.lstart, l_end = tk.lend;
  int cur[2] = {-1, -1};
  int sidx = 0;
  while (sidx < D->nseg && D->seg[sidx].hi < l_start) ++sidx;
  int l = l_start;
  int buf = 0;

  for (; sidx < D->nseg; ++sidx) {
    const int slo = D->seg[sidx].lo, shi = D->seg[sidx].hi;
    if (slo > l_end) break;
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      const int jn = D->seg[sidx].j[s];
      if (jn != cur[s]) {
        if (!SYN) {
          if (cur[s] >= 0) {
            // ---- analysis epilogue: gamma step, write Y^j ----
            const int Lj = D->Lj[cur[s]];
            cx<T>* __restrict__ Y = D->Y[cur[s]];
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int mp = mpb + e;
              if (mp < Lj && m < Lj) {
#pragma unroll
                for (int g = 0; g < N; ++g) {
                  cx<T> v = mkc<T>(0, 0);
#pragma unroll
                  for (int k = 0; k < N; ++k) v = cadd<T>(v, cmul<T>(acc[e][s][k], cgk[k][g]));
                  Y[((size_t)g * Lj + mp) * Lj + m] = cmul_ipow<T>(v, (-m) & 3);
                }
              }
#pragma unroll
              for (int k = 0; k < N; ++k) acc[e][s][k] = mkc<T>(0, 0);
            }
          }
        } else {
          // ---- synthesis prologue: gamma adjoint, load H^j ----
#pragma unroll
          for (int e = 0; e < E; ++e)
#pragma unroll
            for (int k = 0; k < N; ++k) acc[e][s][k] = mkc<T>(0, 0);
          if (jn >= 0) {
            const int Lj = D->Lj[jn];
            const cx<T>* __restrict__ V = D->Y[jn];
#pragma unroll
            for (int e = 0; e < E; ++e) {
              const int mp = mpb + e;
              if (mp < Lj && m < Lj) {
#pragma unroll
                for (int g = 0; g < N; ++g) {
                  const cx<T> vg = V[((size_t)g * Lj + mp) * Lj + m];
#pragma unroll
                  for (int k = 0; k < N; ++k) acc[e][s][k] = cadd<T>(acc[e][s][k], cmul<T>(vg, cgk[k][g]));
                }
#pragma unroll
                for (int k = 0; k < N; ++k) acc[e][s][k] = cmul_ipow<T>(acc[e][s][k], m & 3);
              }
            }
          }
        }
        cur[s] = jn;
      }
    }
    const int lhi = min(shi, l_end);
    for (; l <= lhi; ++l) {
      const bool valid = (m <= l) && (mpb <= l);
      cx<T> part = mkc<T>(0, 0);
      if (valid) {
        const int cl = (l >> 2) + 1;
        const T* __restrict__ slab = delta + delta_slab_offset(l);
        T dv[E];
        if (!tr) {
#pragma unroll
          for (int e = 0; e < E; ++e) dv[e] = __ldg(slab + dA[e] + dB[e] * cl);
        } else {
          VecLd<T, E>::ld(slab + dA[0] + dB[0] * cl, dv);
#pragma unroll
          for (int e = 0; e < E; ++e) dv[e] *= (e & 1) ? -sg0 : sg0;
        }
        const T* __restrict__ rrow = RS + (size_t)l * (NSLOT * N) * Lp + mpb;
        if (!SYN) {
          const cx<T> fv = ldc<T>(f + l * l + l + m);
          cx<T> t[E];
#pragma unroll
          for (int e = 0; e < E; ++e) t[e] = mkc<T>(dv[e] * fv.x, dv[e] * fv.y);
#pragma unroll
          for (int s = 0; s < NSLOT; ++s) {
            if (cur[s] < 0) continue;
#pragma unroll
            for (int k = 0; k < N; ++k) {
              T r[E];
              VecLd<T, E>::ld(rrow + (size_t)(s * N + k) * Lp, r);
#pragma unroll
              for (int e = 0; e < E; ++e) {
                acc[e][s][k].x = fma(t[e].x, r[e], acc[e][s][k].x);
                acc[e][s][k].y = fma(t[e].y, r[e], acc[e][s][k].y);
              }
            }
          }
        } else {
          cx<T> p[E];
#pragma unroll
          for (int e = 0; e < E; ++e) p[e] = mkc<T>(0, 0);
#pragma unroll
          for (int s = 0; s < NSLOT; ++s) {
            if (cur[s] < 0) continue;
#pragma unroll
            for (int k = 0; k < N; ++k) {
              T r[E];
              VecLd<T, E>::ld(rrow + (size_t)(s * N + k) * Lp, r);
#pragma unroll
              for (int e = 0; e < E; ++e) {
                p[e].x = fma(acc[e][s][k].x, r[e], p[e].x);
                p[e].y = fma(acc[e][s][k].y, r[e], p[e].y);
              }
            }
          }
#pragma unroll
          for (int e = 0; e < E; ++e) {
            part.x = fma(dv[e], p[e].x, part.x);
            part.y = fma(dv[e], p[e].y, part.y);
          }
        }
      }
      if (SYN) {
        const int lc = (l - l_start) % LCH;
        red[buf][lc][rg][c] = part;
        if (lc == LCH - 1 || l == l_end) {
          __syncthreads();
          const int lc2 = threadIdx.x >> 5, c2 = threadIdx.x & 31;
          if (lc2 <= lc) {
            cx<T> sum = mkc<T>(0, 0);
#pragma unroll
            for (int r2 = 0; r2 < RG; ++r2) sum = cadd<T>(sum, red[buf][lc2][r2][c2]);
            const int lrow = l - lc + lc2;
            D->P[((size_t)tk.bmp * D->L + lrow) * D->Lp32 + m0 + c2] = sum;
          }
          buf ^= 1;
        }
      }
    }
  }
  if (!SYN) {
#pragma unroll
    for (int s = 0; s < NSLOT; ++s) {
      if (cur[s] < 0) continue;
      const int Lj = D->Lj[cur[s]];
      cx<T>* __restrict__ Y = D->Y[cur[s]];
#pragma unroll
      for (int e = 0; e < E; ++e) {
        const int mp = mpb + e;
        if (mp < Lj && m < Lj) {
#pragma unroll
          for (int g = 0; g < N; ++g) {
            cx<T> v = mkc<T>(0, 0);
#pragma unroll
            for (int k = 0; k < N; ++k) v = cadd<T>(v, cmul<T>(acc[e][s][k], cgk[k][g]));
            Y[((size_t)g * Lj + mp) * Lj + m] = cmul_ipow<T>(v, (-m) & 3);
          }
        }
      }
    }
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
  const T fac = (T)((2.0 * l + 1.0) / (8.0 * 3.14159265358979323846 * 3.14159265358979323846));
  sum = cscale<T>(sum, fac);
  cx<T>* __restrict__ out = reinterpret_cast<cx<T>*>(jobs.out[job]);
  out[l * l + l + m] = sum;
  if (m > 0) {
    const cx<T> cj = cconj<T>(sum);
    out[l * l + l - m] = (m & 1) ? mkc<T>(-cj.x, -cj.y) : cj;
  }
}

template <typename T, int E>
void launch_contract_impl(int N, int nslot, bool syn, const ContractDesc<T>* descs, const TileTask* tiles,
                          int ntiles, const CallPtrs& ptrs, cudaStream_t st) {
  if (ntiles <= 0) return;
  dim3 grid(ntiles), block(256);
#define S2DW_CASE(NN)                                                                          \
  case NN:                                                                                     \
    if (syn) k_contract<T, NN, 2, true, E><<<grid, block, 0, st>>>(descs, tiles, ptrs);        \
    else k_contract<T, NN, 2, false, E><<<grid, block, 0, st>>>(descs, tiles, ptrs);           \
    break;
  if (N == 1 && nslot == 1) {
    if (syn) k_contract<T, 1, 1, true, E><<<grid, block, 0, st>>>(descs, tiles, ptrs);
    else k_contract<T, 1, 1, false, E><<<grid, block, 0, st>>>(descs, tiles, ptrs);
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
