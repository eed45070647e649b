// Direct alpha sums of the small-band scales on the tensor cores (FP32 plans).
//
// Analysis (Eq. (30)), per row (g, b) of X_g[b][m] (m < L_j, complex, stored
// as 2 L_j floats x_k = (Re X_0, Im X_0, Re X_1, ...)):
//   W[row][a] = Re X_0 + 2 sum_{m>=1} Re(X_m e^{i m alpha_a}) = sum_k x_k B[a][k],
//   B[a][2m] = c_m cos(m alpha_a), B[a][2m+1] = -c_m sin(m alpha_a), c_0 = 1, c_m = 2,
// a matrix product with K = 2 L_j <= 64.  Tile: D[a (128)][row (128)] =
// B[a][k] x[row][k]^T in TMEM, so that a warp's TMEM load gives 32
// consecutive samples a of each row and every store is one 128-byte line.
// Synthesis (Eq. (37)): V[row][m] = (2 pi/n) sum_{a<n} W[row][a] e^{-i m alpha_a},
// the product D[row (128)][j (2 L_j, padded)] = W[row][a] C[j][a]^T with
// C[2m][a] = (2 pi/n) cos(m alpha_a), C[2m+1][a] = -(2 pi/n) sin(m alpha_a),
// K = n streamed from HBM in chunks of 32 samples.
//
// FP32 accuracy from TF32 MMAs by the three-product split of tc.cuh.  The
// basis operands are built once per plan, already split and laid out as the
// shared-memory images the MMAs read (tc::img_off), and copied with cp.async;
// the X and W operands are split by the threads on their way to shared memory.
#include "czt.cuh"
#include "tc.cuh"

namespace s2dw {

__device__ int g_tc_timeouts;  // bounded waits that gave up (read and reset by the host)

namespace {

constexpr int kTcA = 128;       // analysis: samples a per tile (MMA M)
constexpr int kTcRows = 128;    // analysis: rows per tile (MMA N)
constexpr int kTcChunk = 1024;  // analysis: rows per CTA
constexpr int kTcAnaThreads = 512;
constexpr int kTcM = 128;       // synthesis: rows per CTA (MMA M)
constexpr int kTcKc = 32;       // synthesis: samples per K chunk
constexpr int kSynStages = 3;   // synthesis: shared-memory ring stages

// The shared-memory and TMEM budgets below hold for K8 <= 64 and NP <= 64.
static_assert(kDirectMaxLjAna <= 32 && kDirectMaxLj <= 32, "tensor-core direct alpha sums sized for L_j <= 32");

__host__ __device__ constexpr int ana_k8(int Lj) { return (2 * Lj + 7) & ~7; }
__host__ __device__ constexpr int syn_npad(int Lj) { return 2 * Lj <= 16 ? 16 : (2 * Lj + 15) & ~15; }

__device__ __forceinline__ void cp16(float* sdst, const float* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_u32(sdst)), "l"(gsrc) : "memory");
}

// smem bytes of the analysis kernel for K8 = 64: basis image (hi, lo) and two
// stages of the row image (hi, lo)
constexpr size_t ana_tc_smem() { return (size_t)(2 + 4) * tc::img_floats(kTcRows, 64) * sizeof(float); }
// smem bytes of the synthesis kernel for Npad = 64: three ring stages of
// (W image, basis image) x (hi, lo)
constexpr size_t syn_tc_smem() {
  return (size_t)kSynStages * 2 * (tc::img_floats(kTcM, kTcKc) + tc::img_floats(64, kTcKc)) * sizeof(float);
}

__global__ void __launch_bounds__(kTcAnaThreads, 1) k_alpha_ana_tc(const CztSeg<float>* __restrict__ segs,
                                                                   int nseg, CallPtrs ptrs) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar[2];
  __shared__ uint32_t tbase;
  __shared__ int fail;
  const CztSeg<float> sg = segs[czt_find_seg<float>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, n = 2 * sg.L - 1, K = 2 * Lj, K8 = ana_k8(Lj);
  const int ntile = (n + kTcA - 1) / kTcA;
  const int ta = item % ntile, a0 = ta * kTcA;
  const int nrows = sg.N * sg.nb, rbeg = (item / ntile) * kTcChunk, rend = min(nrows, rbeg + kTcChunk);
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  float* __restrict__ Wb = reinterpret_cast<float*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff;
  if (Lj <= 0) {  // empty scale: W = 0
    for (int r = rbeg; r < rend; ++r)
      for (int c = t; c < kTcA; c += blockDim.x)
        if (a0 + c < n) Wb[(size_t)r * n + a0 + c] = 0.f;
    return;
  }
  const int img = tc::img_floats(kTcRows, K8);  // = img_floats(kTcA, K8)
  float* Ahi = reinterpret_cast<float*>(smem_raw);
  float* Alo = Ahi + img;
  float* Bimg = Alo + img;  // [stage][hi, lo][img]
  const uint32_t mb0 = tc::smem_u32(&mbar[0]), mb1 = tc::smem_u32(&mbar[1]);
  if (t == 0) {
    tc::mbar_init(mb0, 1);
    tc::mbar_init(mb1, 1);
    fail = 0;
  }
  // TMEM: the sums of stage s at column 128 s
  if (w == 0) tc::tmem_alloc(&tbase, 2 * kTcRows);
  // basis image of this sample tile (built per plan, already split)
  {
    const float* src = reinterpret_cast<const float*>(sg.H) + (size_t)ta * 2 * img;
    for (int i = 4 * t; i < 2 * img; i += 4 * kTcAnaThreads) cp16(Ahi + i, src + i);
    asm volatile("cp.async.commit_group;" ::: "memory");
  }
  const int ntr = (rend - rbeg + kTcRows - 1) / kTcRows;  // row tiles of this CTA
  // staging: thread t holds column k = t % KP of rows rl0 + q RS of a row
  // tile (KP = K8 rounded up to a power of two, RS = 512 / KP >= 8 rows), so
  // the image offset is linear in q and a warp reads consecutive k of a row
  const int lk = K8 <= 8 ? 3 : (K8 <= 16 ? 4 : (K8 <= 32 ? 5 : 6));
  const int k = t & ((1 << lk) - 1), rl0 = t >> lk, RS = kTcAnaThreads >> lk, NQ = kTcRows / RS;
  const bool kin = k < K, kst = k < K8;
  const int o0 = kst ? tc::img_off(rl0, k, K8) : 0, oq = (RS / 8) * (K8 / 4) * tc::kLboF;
  const float* __restrict__ X = reinterpret_cast<const float*>(sg.buf_in);
  const size_t rsk = (size_t)RS * K;  // elements between the rows q and q + 1 of a thread
  auto load = [&](int i, float (&xr)[16]) {  // NQ <= 16
    const int r = rbeg + i * kTcRows + rl0;
    const float* src = X + (size_t)r * K + k;
    const int qn = kin ? (rend - r + RS - 1) / RS : 0;  // rows r + q RS < rend exist
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (q < NQ) xr[q] = q < qn ? __ldg(src) : 0.f;
      src += rsk;
    }
  };
  auto store = [&](int stg, const float (&xr)[16]) {
    float* hi = Bimg + (size_t)stg * 2 * img + o0;
    float* lo = hi + img;
    if (kst) {
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        if (q < NQ) {
          float h, l;
          tc::split_tf32(xr[q], h, l);
          hi[q * oq] = h;
          lo[q * oq] = l;
        }
      }
    }
  };
  const uint32_t idesc = tc::idesc_tf32(kTcA, kTcRows);
  const uint64_t kstep = (uint64_t)(tc::img_kstep_bytes(1) >> 4);  // start-address field per K-step
  auto issue = [&](int stg, uint32_t tmem_d) {  // D = (A_hi B_lo + A_lo B_hi) + A_hi B_hi, cross terms first
    const uint64_t aH = tc::smem_desc(tc::smem_u32(Ahi), K8), aL = tc::smem_desc(tc::smem_u32(Alo), K8);
    const uint64_t bH = tc::smem_desc(tc::smem_u32(Bimg + (size_t)stg * 2 * img), K8);
    const uint64_t bL = tc::smem_desc(tc::smem_u32(Bimg + (size_t)stg * 2 * img + img), K8);
    for (int s = 0; s < K8 / 8; ++s) {
      const uint64_t o = kstep * s;
      tc::mma_tf32(tmem_d, aH + o, bL + o, idesc, s > 0);
      tc::mma_tf32(tmem_d, aL + o, bH + o, idesc, 1);
    }
    for (int s = 0; s < K8 / 8; ++s) {
      const uint64_t o = kstep * s;
      tc::mma_tf32(tmem_d, aH + o, bH + o, idesc, 1);
    }
  };
  // row tiles in registers one tile ahead of their store, two buffers used
  // by name (the loop is unrolled by two), so no copy waits on loads in flight
  float xa[16], xb[16];
  load(0, xa);
  if (ntr > 1) load(1, xb);
  store(0, xa);
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  tc::fence_async_smem();
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  if (t == 0) {
    issue(0, tmem);
    tc::mma_commit(mb0);
  }
  int last = 0;  // last row tile whose MMAs were issued
  // epilogue map: warp w holds samples a0 + 32 (w % 4) + lane and rows 32 (w / 4) .. + 31 of a tile
  const int a = a0 + 32 * (w & 3) + lane, cg = 32 * (w >> 2);
  // tile i: fill = the buffer of tile i (stored), reloaded with tile i + 2; use = tile i + 1
  auto step = [&](int i, float (&use)[16], float (&fill)[16]) -> bool {
    const int s = i & 1;
    if (i + 2 < ntr) load(i + 2, fill);
    if (i + 1 < ntr) store(s ^ 1, use);  // stage s ^ 1: tile i - 1 was waited for
    // one thread waits for tile i's MMAs; the barrier below passes it on
    if (t == 0 && !tc::mbar_wait(s ? mb1 : mb0, (i >> 1) & 1, tc::kWaitCycles)) fail = 1;
    tc::fence_async_smem();
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (fail) return false;  // read after the barrier: the same decision in every thread
    if (i + 1 < ntr) {
      if (t == 0) {
        issue(s ^ 1, tmem + (uint32_t)((s ^ 1) * kTcRows));
        tc::mma_commit(s ^ 1 ? mb1 : mb0);
      }
      last = i + 1;
    }
    const int r0 = rbeg + i * kTcRows + cg;
    const uint32_t te = tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)(s * kTcRows + cg);
    float* pw = Wb + (size_t)r0 * n + a;
    {
      float v[32];
      tc::tmem_ld32(te, v);
      // row j at pw + j n: the pointer advances by one row per store, and a
      // full group of 32 rows (all but the last tile) needs no row test
      const int jn = rend - r0;
      if (a < n && jn > 0) {
        float* q = pw;
        if (jn >= 32) {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            __stcs(q, v[j]);  // written once: streaming
            q += n;
          }
        } else {
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < jn) __stcs(q, v[j]);
            q += n;
          }
        }
      }
    }
    tc::fence_before();
    return true;
  };
  for (int i = 0; i < ntr; i += 2) {
    if (!step(i, xb, xa)) break;
    if (i + 1 < ntr && !step(i + 1, xa, xb)) break;
  }
  if (fail && t == 0) {
    atomicAdd(&g_tc_timeouts, 1);
    // the MMAs in flight (the last commit covers all): a second bounded wait before freeing TMEM
    tc::mbar_wait(last & 1 ? mb1 : mb0, (last >> 1) & 1, tc::kWaitCycles);
  }
  __syncthreads();
  if (w == 0) tc::tmem_free(tmem, 2 * kTcRows);
}

// Synthesis, warp-specialised (one CTA of 128 rows per SM):
//   warps 0-7   producers: W chunk c (registers, two chunks ahead) split into
//               the A image of ring stage c % 3, the basis chunk copied into
//               its B image (cp.async, one chunk ahead); arrive on full[stage]
//   warp  16    MMA issuer (one thread): waits full[stage] and tempty[buffer],
//               12 MMAs into TMEM buffer c % 2, commits to empty[stage] and
//               tfull[buffer]
//   warps 8-15  accumulators: wait tfull[buffer], add the chunk's sums (TMEM
//               lanes = rows, half the columns per warp, one TMEM wait per
//               chunk) to FP32 registers, arrive on tempty[buffer]; finally
//               write V
// No CTA-wide barrier inside the K loop; every wait is bounded and a timeout
// in any role stops all of them.
constexpr int kSynProd = 8;                          // producer warps
constexpr int kSynAcc = 8;                            // accumulator warps
constexpr int kSynThreads = (kSynProd + kSynAcc + 1) * 32;  // + the MMA warp

__global__ void __launch_bounds__(kSynThreads, 1) k_alpha_syn_tc(const CztSeg<float>* __restrict__ segs, int nseg,
                                                                 CallPtrs ptrs) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2 * kSynStages + 4];  // full[S], empty[S], tfull[2], tempty[2]
  __shared__ uint32_t tbase;
  __shared__ volatile int fail;
  const CztSeg<float> sg = segs[czt_find_seg<float>(segs, nseg)];
  const int item = blockIdx.x - sg.start;
  const int Lj = sg.Lj, n = 2 * sg.L - 1, NP = syn_npad(Lj);
  const int nrows = sg.N * sg.nb, r0 = item * kTcM, nr = min(kTcM, nrows - r0);
  const int nchunk = (n + kTcKc - 1) / kTcKc;
  const int t = threadIdx.x, w = t >> 5, lane = t & 31;
  const float* __restrict__ Wb =
      reinterpret_cast<const float*>(sg.is_phi ? ptrs.Wphi[sg.job] : ptrs.W[sg.job]) + sg.woff + (size_t)r0 * n;
  cx<float>* __restrict__ V = sg.buf_out + (size_t)r0 * Lj;
  if (Lj <= 0) return;
  const int imgA = tc::img_floats(kTcM, kTcKc), imgB = tc::img_floats(NP, kTcKc);
  const int stage = 2 * (imgA + imgB);  // floats: A hi, A lo, B hi, B lo
  float* base = reinterpret_cast<float*>(smem_raw);
  // TMEM buffer b (chunk parity): the chunk's sums at column NP b
  const int ncols = 2 * NP <= 32 ? 32 : (2 * NP <= 64 ? 64 : 128);
  auto full = [&](int i) { return tc::smem_u32(&bar[i]); };
  auto empty = [&](int i) { return tc::smem_u32(&bar[kSynStages + i]); };
  auto tfull = [&](int b) { return tc::smem_u32(&bar[2 * kSynStages + b]); };
  auto tempty = [&](int b) { return tc::smem_u32(&bar[2 * kSynStages + 2 + b]); };
  if (t == 0) {
    for (int i = 0; i < kSynStages; ++i) {
      tc::mbar_init(full(i), kSynProd * 32);
      tc::mbar_init(empty(i), 1);
    }
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(tfull(b), 1);
      tc::mbar_init(tempty(b), kSynAcc * 32);
    }
    fail = 0;
  }
  if (w == kSynProd) tc::tmem_alloc(&tbase, ncols);
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tbase;
  int last = -1;  // MMA thread: last chunk whose MMAs were issued
  if (w < kSynProd) {
    // ---- producers: rows w + 8 q (q < 16), samples 32 c + lane ----
    const float* __restrict__ basis = reinterpret_cast<const float*>(sg.H);  // [chunk][B hi, B lo]
    // row w + 8 q at wrow + 8 q n; rows w + 8 q < nr exist (q < nq)
    const float* __restrict__ wrow = Wb + (size_t)w * n + lane;
    const size_t n8 = (size_t)8 * n;
    const int nq = (nr - w + 7) >> 3;
    auto load = [&](int c, float (&x)[16]) {
      const bool ain = kTcKc * c + lane < n;
      const float* __restrict__ p = wrow + kTcKc * c;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        x[q] = (ain && q < nq) ? __ldcs(p) : 0.f;  // read once: streaming
        p += n8;
      }
    };
    auto fetch_basis = [&](int c) {  // basis chunk c into the B images of stage c % S
      float* Bhi = base + (size_t)(c % kSynStages) * stage + 2 * imgA;
      const float* src = basis + (size_t)c * 2 * imgB;
      for (int i = 4 * t; i < 2 * imgB; i += 4 * kSynProd * 32) cp16(Bhi + i, src + i);
      asm volatile("cp.async.commit_group;" ::: "memory");
    };
    // W registers two chunks ahead in a ring of three buffers used by name
    // (the loop is unrolled by three), so no copy waits on loads in flight
    auto step = [&](int c, float (&use)[16], float (&fill)[16]) -> bool {
      if (fail) return false;
      const int st = c % kSynStages;
      if (c + 2 < nchunk) load(c + 2, fill);
      if (c + 1 < nchunk) {
        const int c1 = c + 1;
        if (c1 >= kSynStages &&
            !tc::mbar_wait(empty(c1 % kSynStages), (c1 / kSynStages - 1) & 1, tc::kWaitCycles)) {
          fail = 1;
          return false;
        }
        fetch_basis(c1);  // stage of chunk c + 1 is free: its previous chunk's MMAs completed
      }
      float* Ahi = base + (size_t)st * stage;
      float* Alo = Ahi + imgA;
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const int o = tc::img_off(w + 8 * q, lane, kTcKc);
        float h, l;
        tc::split_tf32(use[q], h, l);
        Ahi[o] = h;
        Alo[o] = l;
      }
      if (c + 1 < nchunk)
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // basis chunk c landed (c + 1 may be in flight)
      else
        asm volatile("cp.async.wait_group 0;" ::: "memory");
      tc::fence_async_smem();
      tc::mbar_arrive(full(st));
      return true;
    };
    float b0[16], b1[16], b2[16];
    load(0, b0);
    if (nchunk > 1) load(1, b1);
    fetch_basis(0);
    for (int c = 0; c < nchunk; c += 3) {
      if (!step(c, b0, b2)) break;
      if (c + 1 < nchunk && !step(c + 1, b1, b0)) break;
      if (c + 2 < nchunk && !step(c + 2, b2, b1)) break;
    }
    asm volatile("cp.async.wait_group 0;" ::: "memory");
  } else if (w < kSynProd + kSynAcc) {
    // ---- accumulators: TMEM lanes 32 (w % 4) .. = rows, columns HC h .. + HC of both
    //      halves (h = 0, 1; HC = NP / 2 = 8, 16, 24 or 32) ----
    const int lrow = 32 * (w & 3), h = (w - kSynProd) >> 2, HC = NP / 2;
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      if (fail) {
        ok = false;
        break;
      }
      const int b = c & 1;
      const bool got = tc::mbar_wait(tfull(b), (c >> 1) & 1, tc::kWaitCycles);
      if (!__all_sync(0xffffffffu, got)) {  // warp-uniform: the TMEM loads below are warp-collective
        fail = 1;
        ok = false;
        break;
      }
      tc::fence_after();
      const uint32_t ta = tmem + ((uint32_t)lrow << 16) + (uint32_t)(NP * b + HC * h);
      if (HC == 32) {
        float v[32];
        tc::tmem_ld32(ta, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) acc[j] += v[j];
      } else if (HC == 16) {
        float va[8], vb[8];
        tc::tmem_ld8x2(ta, ta + 8, va, vb);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          acc[j] += va[j];
          acc[8 + j] += vb[j];
        }
      } else {
#pragma unroll
        for (int g = 0; g < 3; ++g) {
          if (8 * g < HC) {
            float v[8];
            tc::tmem_ld8(ta + 8 * g, v);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[8 * g + j] += v[j];
          }
        }
      }
      tc::fence_before();
      tc::mbar_arrive(tempty(b));
    }
    const int r = lrow + lane;
    if (ok && r < nr) {
#pragma unroll
      for (int j = 0; j < 32; j += 2) {
        const int m = (HC * h + j) >> 1;
        if (j < HC && m < Lj) V[(size_t)r * Lj + m] = mkc<float>(acc[j], acc[j + 1]);
      }
    }
  } else if (lane == 0) {
    // ---- MMA issuer ----
    const uint32_t idesc = tc::idesc_tf32(kTcM, NP);
    const uint64_t kstep = (uint64_t)(tc::img_kstep_bytes(1) >> 4);
    for (int c = 0; c < nchunk; ++c) {
      if (fail) break;
      const int st = c % kSynStages, b = c & 1;
      if (!tc::mbar_wait(full(st), (c / kSynStages) & 1, tc::kWaitCycles) ||
          (c >= 2 && !tc::mbar_wait(tempty(b), ((c >> 1) - 1) & 1, tc::kWaitCycles))) {
        fail = 1;
        break;
      }
      tc::fence_after();
      const uint32_t aH = tc::smem_u32(base + (size_t)st * stage), aL = aH + imgA * 4, bH = aL + imgA * 4,
                     bL = bH + imgB * 4;
      const uint32_t dm = tmem + (uint32_t)(NP * b);
      const uint64_t dAH = tc::smem_desc(aH, kTcKc), dAL = tc::smem_desc(aL, kTcKc);
      const uint64_t dBH = tc::smem_desc(bH, kTcKc), dBL = tc::smem_desc(bL, kTcKc);
#pragma unroll
      for (int k = 0; k < kTcKc / 8; ++k) {  // cross terms first, then hi*hi
        const uint64_t o = kstep * k;
        tc::mma_tf32(dm, dAH + o, dBL + o, idesc, k > 0);
        tc::mma_tf32(dm, dAL + o, dBH + o, idesc, 1);
      }
#pragma unroll
      for (int k = 0; k < kTcKc / 8; ++k) {
        const uint64_t o = kstep * k;
        tc::mma_tf32(dm, dAH + o, dBH + o, idesc, 1);
      }
      tc::mma_commit(empty(st));
      tc::mma_commit(tfull(b));
      last = c;
    }
    // after a timeout: a bounded wait for the MMAs in flight before TMEM is released
    if (fail && last >= 0) tc::mbar_wait(tfull(last & 1), (last >> 1) & 1, tc::kWaitCycles);
  }
  __syncwarp();
  tc::fence_before();
  __syncthreads();
  if (fail && t == 0) atomicAdd(&g_tc_timeouts, 1);
  if (w == kSynProd) tc::tmem_free(tmem, ncols);
}

// Basis images.  Analysis: [tile][hi, lo][img_floats(128, K8)], sample a =
// 128 tile + r, column k.  Synthesis: [chunk][hi, lo][img_floats(NP, 32)],
// row j, sample a = 32 chunk + k.  Values from the exact angle
// 2 pi ((m a) mod n) / n in FP64, then split.
__device__ __forceinline__ void put_split(float* hi, float* lo, int o, double v) {
  const float h = tc::to_tf32((float)v);
  hi[o] = h;
  lo[o] = tc::to_tf32((float)(v - (double)h));
}

__global__ void k_tc_basis_ana(float* out, int n, int Lj) {
  const int K8 = ana_k8(Lj), img = tc::img_floats(kTcA, K8);
  const int ntile = (n + kTcA - 1) / kTcA;
  const long long total = (long long)ntile * kTcA * K8;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int tile = (int)(idx / (kTcA * K8)), r = (int)(idx / K8 % kTcA), k = (int)(idx % K8);
    const int a = tile * kTcA + r, m = k >> 1;
    double v = 0.0;
    if (a < n && k < 2 * Lj) {
      const long long u = ((long long)m * a) % n;
      double sn, cs;
      sincospi(2.0 * (double)u / (double)n, &sn, &cs);
      const double cm = m == 0 ? 1.0 : 2.0;
      v = (k & 1) ? -cm * sn : cm * cs;
    }
    float* hi = out + (size_t)tile * 2 * img;
    put_split(hi, hi + img, tc::img_off(r, k, K8), v);
  }
}

__global__ void k_tc_basis_syn(float* out, int n, int Lj, double scale) {
  const int NP = syn_npad(Lj), img = tc::img_floats(NP, kTcKc);
  const int nchunk = (n + kTcKc - 1) / kTcKc;
  const long long total = (long long)nchunk * NP * kTcKc;
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int c = (int)(idx / (NP * kTcKc)), j = (int)(idx / kTcKc % NP), k = (int)(idx % kTcKc);
    const int a = c * kTcKc + k, m = j >> 1;
    double v = 0.0;
    if (a < n && j < 2 * Lj) {
      const long long u = ((long long)m * a) % n;
      double sn, cs;
      sincospi(2.0 * (double)u / (double)n, &sn, &cs);
      v = (j & 1) ? -scale * sn : scale * cs;
    }
    float* hi = out + (size_t)c * 2 * img;
    put_split(hi, hi + img, tc::img_off(j, k, kTcKc), v);
  }
}

// One warp waits, bounded, on an mbarrier that nothing arrives on: the
// failure path of every bounded wait above (give up, count it), on demand.
__global__ void k_wait_probe(long long limit) {
  __shared__ __align__(8) uint64_t mbar;
  const uint32_t mb = tc::smem_u32(&mbar);
  if (threadIdx.x == 0) tc::mbar_init(mb, 1);
  __syncwarp();
  const bool ok = tc::mbar_wait(mb, 0, limit);
  if (!__any_sync(0xffffffffu, ok) && threadIdx.x == 0) atomicAdd(&g_tc_timeouts, 1);
}

}  // namespace

cudaError_t alpha_tc_wait_probe(long long limit, cudaStream_t st) {
  k_wait_probe<<<1, 32, 0, st>>>(limit);
  return cudaGetLastError();
}

size_t alpha_tc_table_floats(int L, int Lj, bool syn) {
  if (Lj <= 0) return 0;
  const int n = 2 * L - 1;
  if (!syn) return (size_t)((n + kTcA - 1) / kTcA) * 2 * tc::img_floats(kTcA, ana_k8(Lj));
  return (size_t)((n + kTcKc - 1) / kTcKc) * 2 * tc::img_floats(syn_npad(Lj), kTcKc);
}

cudaError_t alpha_tc_build_table(float* out, int L, int Lj, bool syn, cudaStream_t st) {
  const size_t nf = alpha_tc_table_floats(L, Lj, syn);
  if (nf == 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(out, 0, nf * sizeof(float), st);  // image pads
  if (e != cudaSuccess) return e;
  const int n = 2 * L - 1;
  if (syn)
    k_tc_basis_syn<<<256, 256, 0, st>>>(out, n, Lj, 2.0 * 3.14159265358979323846 / n);
  else
    k_tc_basis_ana<<<256, 256, 0, st>>>(out, n, Lj);
  return cudaGetLastError();
}

int alpha_tc_items(int L, int rows, bool syn) {
  if (syn) return (rows + kTcM - 1) / kTcM;
  const int n = 2 * L - 1;
  return ((n + kTcA - 1) / kTcA) * ((rows + kTcChunk - 1) / kTcChunk);
}

void launch_alpha_tc(bool syn, const CztSeg<float>* segs, int nseg, int total_items, const CallPtrs& ptrs,
                     cudaStream_t st) {
  if (total_items <= 0) return;
  if (syn)
    k_alpha_syn_tc<<<total_items, kSynThreads, syn_tc_smem(), st>>>(segs, nseg, ptrs);
  else
    k_alpha_ana_tc<<<total_items, kTcAnaThreads, ana_tc_smem(), st>>>(segs, nseg, ptrs);
}

cudaError_t alpha_tc_prepare() {
  cudaError_t e = cudaFuncSetAttribute(k_alpha_ana_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)ana_tc_smem());
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_alpha_syn_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)syn_tc_smem());
}

cudaError_t alpha_tc_timeouts(int* count) {
  int zero = 0;
  cudaError_t e = cudaMemcpyFromSymbol(count, g_tc_timeouts, sizeof(int));
  if (e != cudaSuccess) return e;
  return cudaMemcpyToSymbol(g_tc_timeouts, &zero, sizeof(int));
}

}  // namespace s2dw
