// Plan-time device kernels, all in float64:
//   * kernel values kappa^j(l), Phi_l0 and |s_ln| (Sec. 2.2, Eqs. (11)-(16));
//   * Driscoll-Healy weights q(theta_t) (Sec. 3.1, Eq. (18));
//   * the Wigner table Delta^l_{m'm} = d^l_{m'm}(pi/2) (Sec. 3.2, Eq. (25));
//   * the per-plan R tables and the chirp-z tables.
#include "fft16.cuh"
#include "internal.h"
#include "plan_kernels.h"

namespace s2dw {


// ---------------------------------------------------------------------------
// k_lambda (Eq. (13)) by composite Gauss-Legendre on [max(t,1/lam), 1].
// ---------------------------------------------------------------------------
__device__ double integrand(double u, double lam) {
  const double x = 2.0 * lam / (lam - 1.0) * (u - 1.0 / lam) - 1.0;
  const double d = 1.0 - x * x;
  if (d <= 0.0) return 0.0;
  return exp(-2.0 / d) / u;  // s_lam(u)^2 / u, s(x) = exp(-1/(1-x^2)) (Eq. (12))
}

// int_lo^hi s_lam(u)^2/u du, limits clipped to the support [1/lam, 1], by a
// whole warp: lane i takes panels i, i + 32, ..., then a butterfly sum (every
// lane ends with the same, order-fixed total).  Called with warp-uniform arguments.
__device__ double I_gl(double lo, double hi, double lam, const double* __restrict__ glx,
                       const double* __restrict__ glw, int Q, int P) {
  lo = fmax(lo, 1.0 / lam);
  hi = fmin(hi, 1.0);
  if (lo >= hi) return 0.0;
  const double h = (hi - lo) / P;
  double tot = 0.0;
  for (int p = threadIdx.x & 31; p < P; p += 32) {
    const double a = lo + p * h, b = (p + 1 == P) ? hi : lo + (p + 1) * h;
    const double mid = 0.5 * (a + b), half = 0.5 * (b - a);
    double s = 0.0;
    for (int q = 0; q < Q; ++q) s += glw[q] * integrand(mid + half * glx[q], lam);
    tot += half * s;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
  return tot;
}

__device__ double k_lambda(double t, double lam, double I0, const double* glx, const double* glw, int Q, int P) {
  if (t <= 1.0 / lam) return 1.0;
  if (t >= 1.0) return 0.0;
  return I_gl(t, 1.0, lam, glx, glw, Q, P) / I0;
}

// The normalisation I(1/lam) = int_{1/lam}^1 s_lam(u)^2/u du of Eq. (13), once.
__global__ void k_kappa_norm(double* I0, double lam, const double* glx, const double* glw, int Q, int P) {
  const double v = I_gl(1.0 / lam, 1.0, lam, glx, glw, Q, P);  // one warp
  if (threadIdx.x == 0) *I0 = v;
}

// kap[j][l] = kappa^j(l) = sqrt(k(t/lam) - k(t)), t = lam^j l / L (Eqs. (14)-(15)),
// with the difference evaluated as the single integral
//   k(t/lam) - k(t) = int_{t/lam}^{t} s_lam(u)^2/u du / I(1/lam)   (Eq. (13)),
// free of cancellation near the support edges; phi[l] = sqrt(k(lam^J l / L)) (Eq. (16)).
// Entries whose interval misses the support [1/lam, 1] are exact 0 (or 1) and
// need no quadrature; about (lam + 1) L of the (J + 2) L entries do.  One warp per entry.
__global__ void k_kernel_values(double* kap, double* phi, int L, int J, double lam, const double* glx,
                                const double* glw, int Q, int P, const double* I0p) {
  const int idx = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (idx >= (J + 2) * L) return;  // warp-uniform
  const bool lead = (threadIdx.x & 31) == 0;
  const int j = idx / L, l = idx % L;
  if (j <= J) {
    const double t = pow(lam, (double)j) * l / L;
    const bool empty = fmax(t / lam, 1.0 / lam) >= fmin(t, 1.0);
    const double v = empty ? 0.0 : sqrt(I_gl(t / lam, t, lam, glx, glw, Q, P) / *I0p);
    if (lead) kap[(size_t)j * L + l] = v;
  } else {
    const double t = pow(lam, (double)J) * l / L;
    const double v = (t <= 1.0 / lam || t >= 1.0) ? sqrt(k_lambda(t, lam, 1.0, glx, glw, Q, P))
                                                  : sqrt(k_lambda(t, lam, *I0p, glx, glw, Q, P));
    if (lead) phi[l] = v;
  }
}

// |s_{l,n_k}| = sqrt(2^-gamma C(gamma, (gamma-n)/2)), gamma = gamma_(N,l) (Eq. (11)); s_0n = 0.
__global__ void k_sabs(double* sabs, int L, int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= L * N) return;
  const int l = idx / N, k = idx % N;
  const int n = -(N - 1) + 2 * k;
  double v = 0.0;
  if (l > 0) {
    const int gam = min(N - 1, ((N + l) % 2 == 0) ? l - 1 : l);
    if (abs(n) <= gam && ((gam - n) & 1) == 0) {
      const int kk = (gam - n) / 2;
      double binom = 1.0;
      for (int i = 1; i <= kk; ++i) binom = binom * (gam - kk + i) / i;
      v = sqrt(ldexp(binom, -gam));
    }
  }
  sabs[idx] = v;
}

// psi[j][l][k] = kappa^j(l) eta |s_{l,n_k}| (Eq. (7)); eta = 1 (N odd) or i (N even).
__global__ void k_psi(double2* psi, const double* kap, const double* sabs, int L, int N, int J) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (J + 1) * L * N) return;
  const int k = idx % N, l = (idx / N) % L, j = idx / (N * L);
  const double v = kap[(size_t)j * L + l] * sabs[l * N + k];
  psi[idx] = (N % 2 == 0) ? make_double2(0.0, v) : make_double2(v, 0.0);
}

// q(theta_t) = (2/L) sin(theta_t) sum_{k<L} sin((2k+1) theta_t)/(2k+1), theta_t = pi(2t+1)/(4L).
// One warp per t: lane i sums k = i, i + 32, ..., then a fixed shuffle tree.
__global__ void k_dh_weights(double* q, int L) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= 2 * L) return;  // warp-uniform
  const long long period = 8LL * L;
  double s = 0.0;
  for (int k = lane; k < L; k += 32) {
    const long long p = ((long long)(2 * k + 1) * (2 * t + 1)) % period;
    s += sinpi((double)p / (4.0 * L)) / (2 * k + 1);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) q[t] = 2.0 / L * sinpi((double)(2 * t + 1) / (4.0 * L)) * s;
}

// ---------------------------------------------------------------------------
// Delta table.  Edge Delta^l_{l,m} = (-1)^{l-m} 2^-l sqrt(C(2l, l+m)) kept as
// mantissa * 2^exponent (it underflows double for large l), walked along the
// diagonals (l,m) -> (l+1,m+1) by the ratio (1/2) sqrt(2l(2l-1)/((l+m)(l+m-1))).
// ---------------------------------------------------------------------------
__global__ void k_delta_edge(double* em, int* ee, int Lmax) {
  const int d = blockIdx.x * blockDim.x + threadIdx.x;
  if (d >= Lmax) return;
  double v = 1.0;
  int e = 0;
  for (int i = 1; i <= d; ++i) v *= -sqrt((2.0 * i - 1.0) / (2.0 * i));
  {
    int k;
    v = frexp(v, &k);
    e += k;
  }
  int l = d, m = 0;
  em[(size_t)l * (l + 1) / 2 + m] = v;
  ee[(size_t)l * (l + 1) / 2 + m] = e;
  for (l = d + 1, m = 1; l < Lmax; ++l, ++m) {
    const double num = 2.0 * l * (2.0 * l - 1.0), den = (double)(l + m) * (double)(l + m - 1);
    v *= 0.5 * sqrt(num / den);
    int k;
    v = frexp(v, &k);
    e += k;
    em[(size_t)l * (l + 1) / 2 + m] = v;
    ee[(size_t)l * (l + 1) / 2 + m] = e;
  }
}

// Column recursion (Trapani-Navaza form at beta = pi/2): for fixed column m,
//   sqrt((l+k)(l-k+1)) Delta_{k-1,m} = 2m Delta_{k,m} - sqrt((l-k)(l+k+1)) Delta_{k+1,m},
// run from k = l (the edge) down to 0 on scaled values.  Stores the rows the
// padded eighth-domain layout keeps for this column (k <= 4 floor(m/4) + 3).
__global__ void __launch_bounds__(128) k_delta_slab(double* d64, float* d32, const double* em, const int* ee,
                                                    int l_base) {
  __shared__ double ia[2049];
  __shared__ double cn[2049];
  const int l = l_base + blockIdx.y;
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if ((int)(blockIdx.x * blockDim.x) > l) return;
  for (int k = threadIdx.x + 1; k <= l; k += blockDim.x) {
    const double a = sqrt((double)(l + k) * (double)(l - k + 1));
    const double c = sqrt((double)(l - k) * (double)(l + k + 1));
    ia[k] = 1.0 / a;
    cn[k] = c / a;
  }
  __syncthreads();
  if (m > l) return;
  const int64_t base = delta_slab_offset(l);
  const int kmax = min(l, 4 * (m >> 2) + 3);
  const int cl = (l >> 2) + 1;
  double cur = em[(size_t)l * (l + 1) / 2 + m];
  int e = ee[(size_t)l * (l + 1) / 2 + m];
  double nxt = 0.0;
  auto store = [&](int k, double v) {
    const double val = ldexp(v, e);
    const int64_t idx = base + delta_row_A(k, m) + (int64_t)delta_row_B(k) * cl;
    d64[idx] = val;
    if (d32) d32[idx] = (float)val;
  };
  if (l <= kmax) store(l, cur);
  const double tm = 2.0 * m;
  for (int k = l; k >= 1; --k) {
    double prv = (tm * cur) * ia[k] - cn[k] * nxt;
    if (fabs(prv) > 0x1p+200) {
      prv *= 0x1p-200;
      cur *= 0x1p-200;
      e += 200;
    }
    if (k - 1 <= kmax) store(k - 1, prv);
    nxt = cur;
    cur = prv;
  }
}

__device__ __forceinline__ double delta_lookup(const double* __restrict__ d64, int l, int mp, int m) {
  double s = 1.0;
  if (mp < 0) {
    mp = -mp;
    if ((l + m) & 1) s = -s;  // Delta_{-m',m} = (-1)^{l+m} Delta_{m'm}
  }
  if (m < 0) {
    m = -m;
    if ((l + mp) & 1) s = -s;  // Delta_{m',-m} = (-1)^{l+m'} Delta_{m'm}
  }
  if (m < 4 * (mp >> 2)) {  // Delta_{m'm} = (-1)^{m'-m} Delta_{m m'}
    const int t = mp;
    mp = m;
    m = t;
    if ((m - mp) & 1) s = -s;
  }
  return s * d64[delta_slab_offset(l) + delta_entry(l, mp, m)];
}

// RS[l][s][h][m'] = Delta^l_{m', n_k} kap[js][l] sabs[l][k] for the orders
// n_k >= 0 only, k = N/2 + h, h < (N+1)/2, js = slotj[l][s] (zero if js < 0,
// m' > l or |n_k| > l).  sabs == nullptr means |s| = 1.  The rows of -n_k
// follow from Delta^l_{m',-n} = (-1)^{l+m'} Delta^l_{m'n} and
// |s_{l,-n}| = |s_{ln}| (Eq. (11) is symmetric in n), so they are not stored.
template <typename T>
__global__ void k_rtable(T* RS, const double* d64, const double* kap, const double* sabs, const int* slotj, int L,
                         int Lp, int N, int nslot, int kapL) {
  const int NH = (N + 1) / 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t total = (int64_t)L * nslot * NH * Lp;
  if (idx >= total) return;
  const int mp = (int)(idx % Lp);
  const int k = N / 2 + (int)((idx / Lp) % NH);
  const int s = (int)((idx / ((int64_t)Lp * NH)) % nslot);
  const int l = (int)(idx / ((int64_t)Lp * NH * nslot));
  const int n = -(N - 1) + 2 * k;
  double v = 0.0;
  const int js = slotj[l * nslot + s];
  if (js >= 0 && mp <= l && abs(n) <= l) {
    const double sa = sabs ? sabs[l * N + k] : 1.0;
    const double kv = kap[(size_t)js * kapL + l];
    if (sa != 0.0 && kv != 0.0) v = delta_lookup(d64, l, mp, n) * kv * sa;
  }
  RS[idx] = (T)v;
}

// Pair table (FP32) of the tile-pair contraction from the FP64 table: block
// (pair (p, q), l) is [r][c] = Delta^l_{32p+r, 32q+c}, zero where an index
// exceeds l.  Grid (Lmax, number of pairs); CTAs with l < 32 q exit.  Each
// thread writes 4 consecutive c (one 16-byte store).
__global__ void __launch_bounds__(256) k_pair_table(float* __restrict__ out, const double* __restrict__ d64,
                                                    int Lmax) {
  const int l = blockIdx.x;
  const int pi = blockIdx.y;
  int q = 0;
  while ((q + 1) * (q + 2) / 2 <= pi) ++q;
  const int p = pi - q * (q + 1) / 2;
  if (l < 32 * q) return;
  const int r = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 4;
  const int mp = 32 * p + r;
  float v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int m = 32 * q + c0 + i;
    v[i] = (mp <= l && m <= l) ? (float)delta_lookup(d64, l, mp, m) : 0.0f;
  }
  float* dst = out + pair_run_base(p, q, Lmax) + (long long)(l - 32 * q) * 1024 + r * 32 + c0;
  *reinterpret_cast<float4*>(dst) = make_float4(v[0], v[1], v[2], v[3]);
}

cudaError_t launch_pair_table(float* out, const double* d64, int Lmax, cudaStream_t st) {
  const int B = Lmax / 32;
  if (B <= 0) return cudaSuccess;
  dim3 grid(Lmax, B * (B + 1) / 2);
  k_pair_table<<<grid, 256, 0, st>>>(out, d64, Lmax);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the read-ahead padding after the last run
  return cudaMemsetAsync(out + pair_run_base(0, B, Lmax), 0, (size_t)kPairPadL * 1024 * sizeof(float), st);
}

// R rows in the layout of the tile-pair contraction:
// RSp[b][l][s][h][c] = R at (l, m' = 32 b + c, slot s, order n_k, k = N/2 + h),
// as k_rtable (zero for l >= L, m' > l, inactive slots).
__global__ void k_rtable_pair(float* RSp, const double* d64, const double* kap, const double* sabs, const int* slotj,
                              int L, int Lr, int N, int nslot, int kapL, int64_t total) {
  const int NH = (N + 1) / 2;
  const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= total) return;
  const int c = (int)(idx & 31);
  const int h = (int)((idx >> 5) % NH);
  const int s = (int)((idx / (32 * NH)) % nslot);
  const int l = (int)((idx / ((int64_t)32 * NH * nslot)) % Lr);
  const int b = (int)(idx / ((int64_t)32 * NH * nslot * Lr));
  const int mp = 32 * b + c;
  const int k = N / 2 + h;
  const int n = -(N - 1) + 2 * k;
  double v = 0.0;
  if (l < L) {
    const int js = slotj[l * nslot + s];
    if (js >= 0 && mp <= l && abs(n) <= l) {
      const double sa = sabs ? sabs[l * N + k] : 1.0;
      const double kv = kap[(size_t)js * kapL + l];
      if (sa != 0.0 && kv != 0.0) v = delta_lookup(d64, l, mp, n) * kv * sa;
    }
  }
  RSp[idx] = (float)v;
}

cudaError_t launch_rtable_pair(float* RSp, const double* d64, const double* kap, const double* sabs,
                               const int* slotj, int L, int Lr, int N, int nslot, int kapL, cudaStream_t st) {
  const int nb = (L + 31) / 32;
  const int64_t total = (int64_t)nb * Lr * nslot * ((N + 1) / 2) * 32;
  if (total == 0) return cudaSuccess;
  k_rtable_pair<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(RSp, d64, kap, sabs, slotj, L, Lr, N, nslot, kapL, total);
  return cudaGetLastError();
}

// Entry i of the twiddle table of length 2^logM: locate level d, then (k, j)
// in it: e^{-2 pi i j k / S_d}.
template <typename T>
__device__ __forceinline__ cx<T> twiddle_entry(int i, int logM) {
  const int M = 1 << logM;
  int d = 0, off = 0;
  while (i >= off + 15 * (M >> (4 * (d + 1)))) {
    off += 15 * (M >> (4 * (d + 1)));
    ++d;
  }
  const int Q = M >> (4 * (d + 1)), S = 16 * Q;
  const int k = (i - off) / Q + 1, j = (i - off) % Q;
  const long long p = ((long long)j * k) % S;
  double s, c;
  sincospi(-2.0 * (double)p / S, &s, &c);
  return mkc<T>((T)c, (T)s);
}

__global__ void k_twiddles(double2* tw, int logM) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < fft_twiddle_entries(logM)) tw[i] = twiddle_entry<double>(i, logM);
}

// Kernels of the segmented chirp-z (segment s = blockIdx.y starts at sample
// a_s = s P), natural order mod M, float64:
//   analysis  h_s[d] = e^{-i pi (d + a_s)^2 / n}, d in [-(Lj-1), M - Lj];
//   synthesis g_s[d] = e^{+i pi (d - a_s)^2 / n}, d in [-(Lj+P-2), M - Lj - P + 1].
__global__ void k_seg_kernels(double2* Ha, double2* Hs, int L, int Lj, int M, int P) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int s = blockIdx.y;
  if (v >= M) return;
  const long long n = 2LL * L - 1, as = (long long)s * P;
  double sn, cs;
  {
    const long long u0 = -(long long)(Lj - 1);
    const long long d = u0 + ((((long long)v - u0) % M) + M) % M;
    const long long e = d + as, p = ((e % (2 * n)) * (e % (2 * n))) % (2 * n);
    sincospi((double)p / (double)n, &sn, &cs);
    Ha[(size_t)s * M + v] = make_double2(cs, -sn);
  }
  {
    const long long u0 = -(long long)(Lj + P - 2);
    const long long d = u0 + ((((long long)v - u0) % M) + M) % M;
    long long e = (d - as) % (2 * n);
    if (e < 0) e += 2 * n;
    const long long p = (e * e) % (2 * n);
    sincospi((double)p / (double)n, &sn, &cs);
    Hs[(size_t)s * M + v] = make_double2(cs, sn);
  }
}

// Chirp tables (angles reduced exactly in integers before sincospi).
template <typename T>
__global__ void k_chirp_tables(cx<T>* tw, cx<T>* chirp_a, cx<T>* pre_b, cx<T>* post_b, cx<T>* preS_b,
                               cx<T>* postS_b, cx<T>* root_a, cx<T>* bfft, const double* q, int L, int logM) {
  const int M = 1 << logM;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int n = 2 * L - 1;
  double s, c;
  if (i < fft_twiddle_entries(logM)) tw[i] = twiddle_entry<T>(i, logM);
  if (i < n) {
    const long long p = ((long long)i * i) % (2LL * n);
    sincospi((double)p / n, &s, &c);
    chirp_a[i] = mkc<T>((T)c, (T)s);
    sincospi(2.0 * i / n, &s, &c);  // roots of unity e^{2 pi i t/n} for the direct alpha sums
    root_a[i] = mkc<T>((T)c, (T)s);
  }
  if (i < 2 * L - 1) {
    const long long mp = (long long)i - (L - 1);
    const long long p = (mp * (mp + 1)) % (8LL * L);
    sincospi((double)p / (4.0 * L), &s, &c);
    pre_b[i] = mkc<T>((T)c, (T)s);
    postS_b[i] = mkc<T>((T)c, (T)(-s));
    sincospi((double)mp / (4.0 * L), &s, &c);  // e^{i pi m'/(4L)}: shift of the beta grid
    bfft[i] = mkc<T>((T)c, (T)s);
  }
  if (i < 2 * L) {
    const long long p = ((long long)i * i) % (8LL * L);
    sincospi((double)p / (4.0 * L), &s, &c);
    post_b[i] = mkc<T>((T)c, (T)s);
    preS_b[i] = mkc<T>((T)(q[i] * c), (T)(-q[i] * s));
    bfft[2 * L - 1 + i] = mkc<T>((T)q[i], (T)0);
  }
}

// Chirp kernels h_u at u mod M, natural order, float64: kinds 0..3 =
// beta ana (e^{-i pi u^2/(4L)}, u0 = -(L-1)), alpha ana (e^{-i pi u^2/n}, u0 = -(L-1)),
// alpha syn (e^{+i pi u^2/n}, u0 = L-M), beta syn (e^{+i pi u^2/(4L)}, u0 = L-M).
__global__ void k_chirp_kernels(double2* H, int L, int M) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  const int kind = blockIdx.y;
  if (v >= M) return;
  const int n = 2 * L - 1;
  const long long u0 = (kind < 2) ? -(long long)(L - 1) : (long long)L - M;
  const long long u = u0 + ((((long long)v - u0) % M) + M) % M;
  const long long period = (kind == 0 || kind == 3) ? 8LL * L : 2LL * n;
  const double denom = (kind == 0 || kind == 3) ? 4.0 * L : (double)n;
  const long long p = (u * u) % period;
  double s, c;
  sincospi((double)p / denom, &s, &c);
  const double sign = (kind < 2) ? -1.0 : 1.0;
  H[(size_t)kind * M + v] = make_double2(c, sign * s);
}

// Spectrum of each chirp kernel: the forward stages of the convolution engine
// (its digit-reversed order), scaled by 1/M, stored for the innermost stage:
// entry k of block u (position u R + k, R its radix) at k (M/R) + u, so that
// the R loads of a thread are each coalesced across the warp.
__global__ void __launch_bounds__(256) k_chirp_spectra(double2* H, const double2* tw, int logM) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double2* A = reinterpret_cast<double2*>(smem_raw);
  const int M = 1 << logM;
  double2* h = H + (size_t)blockIdx.x * M;
  for (int v = threadIdx.x; v < M; v += blockDim.x) A[fpad(v)] = h[v];
  __syncthreads();
  fft_forward_inplace<double>(A, logM, tw, 1.0 / M);
  int R, nmid;
  fft_schedule(logM, R, nmid);
  const int nb = M / R;
  for (int v = threadIdx.x; v < M; v += blockDim.x) h[(v % R) * nb + v / R] = A[fpad(v)];
}

template <typename T>
__global__ void k_to_prec(cx<T>* dst, const double2* src, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = mkc<T>((T)src[i].x, (T)src[i].y);
}

// ---------------------------------------------------------------------------
// Host launchers
// ---------------------------------------------------------------------------
static inline unsigned nblk(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

cudaError_t launch_kernel_values(double* kap, double* phi, double* sabs, double2* psi, double* q, int L, int N,
                                 int J, double lam, const double* glx, const double* glw, int Q, int P,
                                 double* I0, cudaStream_t st) {
  k_kappa_norm<<<1, 32, 0, st>>>(I0, lam, glx, glw, Q, P);
  k_kernel_values<<<nblk((int64_t)(J + 2) * L * 32, 128), 128, 0, st>>>(kap, phi, L, J, lam, glx, glw, Q, P, I0);
  k_sabs<<<nblk((int64_t)L * N, 128), 128, 0, st>>>(sabs, L, N);
  k_psi<<<nblk((int64_t)(J + 1) * L * N, 128), 128, 0, st>>>(psi, kap, sabs, L, N, J);
  return launch_dh_weights(q, L, st);
}

cudaError_t launch_dh_weights(double* q, int L, cudaStream_t st) {
  k_dh_weights<<<nblk(2 * (int64_t)L * 32, 128), 128, 0, st>>>(q, L);
  return cudaGetLastError();
}

cudaError_t launch_delta_build(double* d64, float* d32, double* em, int* ee, int Lmax, int l_first,
                               cudaStream_t st) {
  // one thread per diagonal, each a serial FP64 chain: 32 threads per CTA
  // spread the chains over as many SMs as possible
  k_delta_edge<<<nblk(Lmax, 32), 32, 0, st>>>(em, ee, Lmax);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  // slabs l_first .. Lmax-1 in chunks of l so that a single launch stays short
  const int chunk = 256;
  for (int l0 = l_first; l0 < Lmax; l0 += chunk) {
    const int nl = (Lmax - l0 < chunk) ? Lmax - l0 : chunk;
    dim3 grid(nblk(l0 + nl, 128), nl);
    k_delta_slab<<<grid, 128, 0, st>>>(d64, d32, em, ee, l0);
    err = cudaGetLastError();
    if (err != cudaSuccess) return err;
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_rtable(T* RS, const double* d64, const double* kap, const double* sabs, const int* slotj, int L,
                          int Lp, int N, int nslot, int kapL, cudaStream_t st) {
  const int64_t total = (int64_t)L * nslot * ((N + 1) / 2) * Lp;
  if (total == 0) return cudaSuccess;
  k_rtable<T><<<nblk(total, 256), 256, 0, st>>>(RS, d64, kap, sabs, slotj, L, Lp, N, nslot, kapL);
  return cudaGetLastError();
}

// The shared-memory limit of k_chirp_spectra, set to that of the longest
// transform (M = 2^13, L <= 2048) whatever the call's length: plans built
// concurrently in several host threads then never lower the limit between
// another thread's setting and its launch.
cudaError_t chirp_spectra_prepare() {
  return cudaFuncSetAttribute(k_chirp_spectra, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(double2) * fft_smem_elems(1 << 13));
}

cudaError_t launch_chirp_build64(double2* tw, double2* chirp_a, double2* pre_b, double2* post_b, double2* preS_b,
                                 double2* postS_b, double2* root_a, double2* bfft, double2* H, const double* q, int L,
                                 int logM,
                                 cudaStream_t st) {
  const int M = 1 << logM;
  const int cnt = (M > 2 * L) ? M : 2 * L;
  k_chirp_tables<double><<<nblk(cnt, 256), 256, 0, st>>>(tw, chirp_a, pre_b, post_b, preS_b, postS_b, root_a, bfft,
                                                         q, L, logM);
  k_chirp_kernels<<<dim3(nblk(M, 256), 4), 256, 0, st>>>(H, L, M);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int smem = (int)sizeof(double2) * fft_smem_elems(M);
  err = chirp_spectra_prepare();
  if (err != cudaSuccess) return err;
  k_chirp_spectra<<<4, 256, smem, st>>>(H, tw, logM);
  return cudaGetLastError();
}

int twiddle_entries(int logM) { return fft_twiddle_entries(logM); }

cudaError_t launch_twiddles64(double2* tw, int logM, cudaStream_t st) {
  const int n = fft_twiddle_entries(logM);
  if (n <= 0) return cudaSuccess;
  k_twiddles<<<nblk(n, 256), 256, 0, st>>>(tw, logM);
  return cudaGetLastError();
}

// MW beta chirp: pre_mw[m' + L - 1] = e^{i pi (m'^2 + m')/n}, |m'| < L, n = 2L-1
// (the linear term is the grid's offset beta_b = (2b+1) pi / n).
__global__ void k_mw_pre(double2* pre, int L) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const long long n = 2LL * L - 1;
  if (i >= n) return;
  const long long mp = (long long)i - (L - 1);
  long long p = (mp * (mp + 1)) % (2 * n);
  if (p < 0) p += 2 * n;
  double s, c;
  sincospi((double)p / (double)n, &s, &c);
  pre[i] = make_double2(c, s);
}

cudaError_t launch_mw_pre64(double2* pre, int L, cudaStream_t st) {
  k_mw_pre<<<nblk(2 * (int64_t)L - 1, 256), 256, 0, st>>>(pre, L);
  return cudaGetLastError();
}

cudaError_t launch_seg_build64(double2* tw, double2* Ha, double2* Hs, int L, int Lj, int logM, int P, int S,
                               cudaStream_t st) {
  const int M = 1 << logM;
  k_twiddles<<<nblk(fft_twiddle_entries(logM), 256), 256, 0, st>>>(tw, logM);
  k_seg_kernels<<<dim3(nblk(M, 256), S), 256, 0, st>>>(Ha, Hs, L, Lj, M, P);
  cudaError_t err = cudaGetLastError();
  if (err != cudaSuccess) return err;
  const int smem = (int)sizeof(double2) * fft_smem_elems(M);
  err = chirp_spectra_prepare();
  if (err != cudaSuccess) return err;
  k_chirp_spectra<<<S, 256, smem, st>>>(Ha, tw, logM);
  k_chirp_spectra<<<S, 256, smem, st>>>(Hs, tw, logM);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_to_prec(cx<T>* dst, const double2* src, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_to_prec<T><<<nblk(n, 256), 256, 0, st>>>(dst, src, n);
  return cudaGetLastError();
}

template cudaError_t launch_rtable<float>(float*, const double*, const double*, const double*, const int*, int, int,
                                          int, int, int, cudaStream_t);
template cudaError_t launch_rtable<double>(double*, const double*, const double*, const double*, const int*, int,
                                           int, int, int, int, cudaStream_t);
template cudaError_t launch_to_prec<float>(float2*, const double2*, int64_t, cudaStream_t);

// Timing inputs: a 32-bit integer hash (multiply-xorshift rounds) of the
// index, scaled to [-1/2, 1/2).  Only the run time of the transforms that read
// these values matters, not their distribution.
template <typename T>
__global__ void k_fill_noise(T* __restrict__ dst, int64_t n, uint32_t seed) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)i * 0x9E3779B1u ^ seed ^ (uint32_t)(i >> 32) * 0x85EBCA77u;
    h ^= h >> 15;
    h *= 0x2C1B3C6Du;
    h ^= h >> 12;
    h *= 0x297A2D39u;
    h ^= h >> 15;
    dst[i] = (T)((double)h * (1.0 / 4294967296.0) - 0.5);
  }
}

template <typename T>
cudaError_t launch_fill_noise(T* dst, int64_t n, uint32_t seed, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
  k_fill_noise<T><<<(unsigned)blocks, 256, 0, st>>>(dst, n, seed);
  return cudaGetLastError();
}
template cudaError_t launch_fill_noise<float>(float*, int64_t, uint32_t, cudaStream_t);
template cudaError_t launch_fill_noise<double>(double*, int64_t, uint32_t, cudaStream_t);

}  // namespace s2dw
