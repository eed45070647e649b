/*
 * s2dw.h -- C ABI of the GB300 directional scale-discretized wavelet transform.
 *
 * The transform is the one of McEwen, Vandergheynst & Wiaux, "On the
 * computation of directional scale-discretized wavelet transforms on the
 * sphere" (2013):
 *   analysis  W^j(alpha,beta,gamma) = sum_{l<L,m,n} f_lm Psi^j*_ln D^l*_mn
 *             (Sec. 3.2, Eq. (20)), scaling coefficients W^Phi (Eqs. (3), (31));
 *   synthesis f_lm from W^j and W^Phi (Sec. 3.3, Eqs. (32)-(41)),
 * both exact on the Driscoll-Healy SO(3) grid of Sec. 3.1 and computed by the
 * factoring of rotations (Eq. (25)) and a separation of variables.
 *
 * Conventions shared by every entry point:
 *   - Signals are real on the sphere: f_{l,-m} = (-1)^m conj(f_lm).  Analysis
 *     reads only m >= 0; synthesis writes every m (m < 0 by that symmetry).
 *   - f_lm: flat array indexed l*l + l + m, |m| <= l < L.
 *   - W:  real array [J+1][N][2L][2L-1] = [scale j][gamma_g][beta_b][alpha_a],
 *         alpha_a = 2 pi a/(2L-1), beta_b = pi (2b+1)/(4L), gamma_g = pi g/N
 *         (Sec. 3.1).  Scale j = 0 is the finest.
 *   - Wphi: real array [2L][2L-1] = [theta_t][phi_p] on the same grid.
 *   - S2DW_MW plans sample beta at the L values beta_b = pi (2b+1)/(2L-1),
 *     b < L (the McEwen-Wiaux grid, Sec. 4): every 2L above is then L.
 *   - Precision: S2DW_FP64 plans take complex128 f and double W / Wphi;
 *     S2DW_MIXED plans take complex64 f and float W / Wphi (FP32 arithmetic,
 *     Wigner Delta generated in FP64 and stored in FP32).
 *   - Ownership: the caller owns every f / W / Wphi buffer; the plan owns its
 *     device workspace; the process owns the shared Delta table (reference
 *     counted, freed with the last plan).
 *   - Device buffers must be 16-byte aligned (cudaMalloc / torch give 256).
 *   - Calls are asynchronous on `stream` (a cudaStream_t, NULL = legacy
 *     default stream); they never synchronise the device except where noted.
 *   - Every entry point returns S2DW_OK (0) or a negative status; nothing
 *     throws or exits across the ABI.  s2dw_strerror gives static text.
 *   - A plan must not run two calls concurrently (its workspace is shared
 *     between calls); use one plan per stream for concurrency.
 */
#ifndef S2DW_H
#define S2DW_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  S2DW_OK = 0,
  S2DW_EINVAL = -1,   /* invalid argument (sizes, flags, NULL pointers)   */
  S2DW_ENOMEM = -2,   /* device allocation failed                          */
  S2DW_ECUDA = -3,    /* a CUDA call or kernel launch failed               */
  S2DW_ETIMEOUT = -4, /* a bounded device wait ran out                     */
  S2DW_EBUSY = -5,    /* resource in use                                   */
  S2DW_ENOTSUP = -6   /* valid request outside what this build supports    */
};

enum {
  S2DW_FP64 = 1,        /* plain float64 path                              */
  S2DW_MIXED = 2,       /* float32 arithmetic, FP64-generated Delta        */
  S2DW_REAL_SIGNAL = 4, /* real signals (required; set implicitly)         */
  S2DW_MULTIRES = 8,    /* each scale on the grid of its own band-limit     */
  S2DW_MW = 16          /* L beta samples (McEwen-Wiaux grid), not 2L       */
};

typedef struct s2dw_plan_s* s2dw_plan_t;

/*
 * s2dw_plan: create a plan for band-limit L, azimuthal band-limit N,
 * dilation lambda and J0.
 *   Scales: J_max = ceil(log_lambda L) (Sec. 2.2), J = J_max - J0, wavelet
 *   scales j = 0..J; the scaling function Phi covers the rest (Eq. (16)).
 *   Kernels: Psi^j_ln = kappa^j(l) s_ln (Eqs. (7), (11)-(15)).
 * Valid requests: L >= 2, 1 <= N <= L, lambda > 1 (finite), 0 <= J0 <= J_max;
 * flags = exactly one of S2DW_FP64 / S2DW_MIXED, optionally | S2DW_REAL_SIGNAL
 * and | one of S2DW_MULTIRES / S2DW_MW.  Otherwise S2DW_EINVAL.
 * Limits of this build: L <= 2048, N <= 8 and at most 64 scales (J + 1);
 * a valid request beyond them returns S2DW_ENOTSUP.
 * S2DW_MULTIRES samples each W^j on the DH SO(3) grid of its own band-limit
 * L_j = 1 + the largest l with kappa^j(l) > 0 (and W^Phi on the sphere grid
 * of L_Phi): W^j is band-limited there, so the samples are exact and the
 * synthesis stays exact, with fewer samples and less work (the paper notes
 * that not every scale needs the full band-limit, Sec. 3.2).  W is then one
 * array holding the scales one after the other (s2dw_scale_grid gives each
 * scale's band-limit, offset and size).
 * S2DW_MW samples beta at beta_b = pi (2b+1)/(2L-1), b < L, the grid whose
 * sampling theorem Sec. 4 names as the replacement of the DH grid: half the
 * beta samples (the last is beta = pi), alpha and gamma as in Sec. 3.1.
 * Analysis evaluates Eq. (20) / Eq. (3) there.  Synthesis is exact for the
 * coefficients of a band-limited signal: per Fourier component (m, n) the
 * beta dependence is a trigonometric polynomial of degree < L_j with
 * U(2 pi - beta) = (-1)^{m-n} U(beta), so the L samples and their
 * reflections are 2L-1 equispaced torus samples; its coefficients are taken
 * from them (the self-reflected sample beta = pi weighted (1 + (-1)^{m-n})/2),
 * evaluated on the DH beta grid and the DH synthesis of Sec. 3.3 follows.
 * For arbitrary arrays this synthesises their projection onto that space.
 * Work: evaluates the kernels, the DH weights (Eq. (18)) and the Delta table
 * on the device (FP64 recursion, grown to cover l < L on first need) and
 * allocates the workspace (stream-ordered, on a private stream; other
 * streams keep running).  Returns once the plan is ready for any stream.
 * *out receives the plan; on failure *out is NULL and nothing leaks.
 */
int s2dw_plan(s2dw_plan_t* out, int L, int N, double lambda, int J0, unsigned flags);

/* Release a plan (NULL is accepted).  Waits only for this plan's last
 * recorded call (not the whole device), then frees its workspace.  Calls
 * captured into a CUDA graph are not tracked: destroy a plan only once no
 * graph that captured it can run again (as for the buffers passed to it). */
int s2dw_plan_destroy(s2dw_plan_t plan);

/*
 * s2dw_query: sizes of a plan, any pointer may be NULL.
 *   J: largest scale index (scales 0..J);
 *   w_elems_per_scale: N * nb * (2L-1), nb = 2L (L for S2DW_MW plans; 0 for
 *   S2DW_MULTIRES plans, whose scales differ in size); wphi_elems:
 *   nb_Phi * (2L_Phi-1), L_Phi = L and nb_Phi = nb unless S2DW_MULTIRES;
 *   workspace_bytes: device bytes owned by the plan (intermediates, tables);
 *   total_device_bytes: workspace_bytes + the caller's f, W, Wphi bytes for
 *   one transform (used for admission by HBM footprint).
 */
int s2dw_query(s2dw_plan_t plan, int* J, int64_t* w_elems_per_scale, int64_t* wphi_elems,
               int64_t* workspace_bytes, int64_t* total_device_bytes);

/*
 * s2dw_scale_grid: sampling grid of scale j (0 <= j <= J) or, for j = J+1,
 * of the scaling part: its band-limit Lg (nb = 2Lg beta samples, Lg for
 * S2DW_MW, and 2Lg-1 alpha samples), the element offset of W^j in W (0 for
 * j = J+1: W^Phi is its own array) and the element count (N nb (2Lg-1), or
 * nb (2Lg-1)).  Any output may be NULL.
 * S2DW_EINVAL for j outside [0, J+1].
 */
int s2dw_scale_grid(s2dw_plan_t plan, int j, int* Lgrid, int64_t* offset, int64_t* elems);

/*
 * s2dw_alpha_method: how the alpha sums of scale j (0 <= j <= J, or J+1 for
 * the scaling part) are evaluated (Eqs. (30), (37)), per direction
 * (dir 0 analysis, 1 synthesis):
 *   *method = 0: direct sums (small band L_j);
 *             1: one chirp-z convolution of length *fft_len over all 2Lg-1
 *                samples (*segments = 1);
 *             2: segmented chirp-z: *segments convolutions of length
 *                *fft_len, each covering *seg_len samples, sharing one
 *                forward FFT (analysis) or one inverse FFT (synthesis).
 * Host only; any output may be NULL.  S2DW_EINVAL for a bad j or dir.
 */
int s2dw_alpha_method(s2dw_plan_t plan, int j, int dir, int* method, int* fft_len, int* segments, int* seg_len);

/*
 * s2dw_launch_counts: number of kernel launches one s2dw_analysis and one
 * s2dw_synthesis call of this plan issue (stages with no work launch
 * nothing).  Either pointer may be NULL.  Host only; no counterpart in the
 * paper (launch accounting of this implementation).
 */
int s2dw_launch_counts(s2dw_plan_t plan, int* analysis, int* synthesis);

/*
 * s2dw_kernels: copy the plan's kernels to HOST memory (synchronous).
 *   psi: complex128 as interleaved doubles [J+1][L][N][2]: Psi^j_{l,n_k},
 *        n_k = -(N-1) + 2k  (Eq. (7));  phi: double [L]: Phi_l0 (Eq. (16)).
 * Either pointer may be NULL.
 */
int s2dw_kernels(s2dw_plan_t plan, double* psi, double* phi);

/*
 * s2dw_analysis: wavelet and scaling coefficients of f (device pointers).
 *   f: [L*L] complex (m >= 0 read);  W: [J+1][N][2L][2L-1] real;
 *   Wphi: [2L][2L-1] real.  Sec. 3.2: the l-contraction into the Fourier
 *   cube (Eq. (27)), then the gamma, beta and alpha sums (Eqs. (28)-(30)).
 */
int s2dw_analysis(s2dw_plan_t plan, const void* flm, void* W, void* Wphi, void* stream);

/*
 * s2dw_synthesis: f_lm from W and Wphi (device pointers; same layouts).
 *   Sec. 3.3: alpha (Eq. (37)), gamma (Eq. (39)), beta (Eq. (40))
 *   quadratures, then the Delta contraction (Eqs. (34), (32)) and the
 *   scaling term (Eq. (41)).  Writes every (l, m).
 */
int s2dw_synthesis(s2dw_plan_t plan, const void* W, const void* Wphi, void* flm, void* stream);

/*
 * Batched forms: njobs (1..64) transforms, each with its own plan (plans may
 * differ in L, N, lambda and J0 but must be distinct objects of one precision;
 * mixed precisions give S2DW_ENOTSUP), run as one set of launches per stage
 * (the contraction once per distinct N).  Arrays are HOST arrays of njobs
 * device pointers.  Same layouts as the single calls.  The launch lists of a
 * plan set are built on first use and cached until one of its plans is
 * destroyed, so repeated batches (e.g. under CUDA graph capture) make no
 * host-to-device copies.
 */
int s2dw_analysis_batch(const s2dw_plan_t* plans, const void* const* flm, void* const* W,
                        void* const* Wphi, int njobs, void* stream);
int s2dw_synthesis_batch(const s2dw_plan_t* plans, const void* const* W, const void* const* Wphi,
                         void* const* flm, int njobs, void* stream);

/*
 * Spherical harmonic transforms of a real signal on the DH sphere grid of
 * Sec. 3.1 (theta_t = pi(2t+1)/(4L), t < 2L; phi_p = 2 pi p/(2L-1)), with
 * Y_lm(theta, phi) = sqrt((2l+1)/(4 pi)) e^{i m phi} d^l_m0(theta) (Sec. 2.1):
 *   s2dw_sht_inverse: fpix[t][p] = sum_{l<L, |m|<=l} f_lm Y_lm(theta_t, phi_p);
 *   s2dw_sht_forward: f_lm = sum_{t,p} q_t (2 pi/(2L-1)) fpix[t][p] Y*_lm, the
 *     DH quadrature of Eqs. (17)-(18), exact for band-limited samples.
 *   flm: device [L*L] complex (index l*l + l + m); fpix: device [2L][2L-1]
 *   real, in the plan's precision.  They let a caller start from pixel
 *   values: W = analysis(sht_forward(f)), f = sht_inverse(synthesis(W)).
 * The first call builds a companion plan (no wavelet scales, Phi_l =
 * sqrt((2l+1)/(4 pi))) on the plan's private stream; later calls are
 * asynchronous on `stream`.  S2DW_EINVAL for NULL pointers.
 */
int s2dw_sht_inverse(s2dw_plan_t plan, const void* flm, void* fpix, void* stream);
int s2dw_sht_forward(s2dw_plan_t plan, const void* fpix, void* flm, void* stream);

/*
 * s2dw_steer: wavelet coefficients at arbitrary orientations from the N
 * sampled ones (steerability, Sec. 2.2 Eq. (10)):
 *   out[j][t][b][a] = sum_{g<N} z(gamma_t - gamma_g) W[j][g][b][a],
 *   z(x) = (1/N) sum_{n in S_N} e^{i n x}, gamma_g = pi g / N (z_n = 1/N,
 *   the even/odd directional kernels of Eq. (11)).
 *   W: device [J+1][N][2L][2L-1] real, as written by s2dw_analysis;
 *   gammas: HOST double[ngamma], any real angles (1 <= ngamma <= 32);
 *   out: device [J+1][ngamma][2L][2L-1] real (the plan's precision); for an
 *   S2DW_MULTIRES plan each scale's [ngamma][2Lg][2Lg-1] block, in order.
 * Asynchronous on stream (one pass over W, HBM-bound).  The scaling
 * coefficients have no orientation and are not involved.
 * S2DW_EINVAL for a NULL pointer or ngamma outside [1, 32].
 */
int s2dw_steer(s2dw_plan_t plan, const void* W, const double* gammas, int ngamma, void* out, void* stream);

/* Static text for a status code (never NULL, never freed by the caller). */
const char* s2dw_strerror(int status);

/*
 * s2dw_wait_timeouts: number of bounded waits in the library's kernels that
 * gave up since the last call (0 in normal operation).  The tensor-core
 * kernels of the small-band alpha sums (FP32 plans) wait on an mbarrier for
 * their matrix products, and the FP32 contraction for the bulk copies of its
 * operands, about one second at most; one that gives up skips the rest of
 * its work (and releases its tensor memory, or waits for its copies in
 * flight), so the output of that call is invalid.  Synchronous (waits for the device); reads and resets the
 * count.  Returns S2DW_ETIMEOUT when the count is nonzero (the count is
 * written either way), S2DW_EINVAL for NULL.
 */
int s2dw_wait_timeouts(int* count);

/*
 * s2dw_wait_probe: the failure path of those waits, on demand.  Launches one
 * warp on `stream` that waits on an mbarrier nothing arrives on, for at most
 * limit_cycles SM cycles (clamped to [1e3, 2e9]), gives up and counts it like
 * any bounded wait of the library: the next s2dw_wait_timeouts reports it.
 * No fault, trap or hang is involved; the context stays usable.
 */
int s2dw_wait_probe(long long limit_cycles, void* stream);

/*
 * Introspection used by the tests (synchronous, host outputs).
 *   s2dw_scale_support: l-range [lo, hi] on which kappa^j(l) > 0 (j = J+1
 *     gives Phi's range, lo = 0).
 *   s2dw_delta_slab: Delta^l_{m'm} = d^l_{m'm}(pi/2) (below Eq. (25)) for
 *     0 <= m', m <= l from the FP64 table, into a host [l+1][l+1] array;
 *     requires l < L of the plan.
 *   s2dw_stage: copy intermediate `stage` of scale j from the last call on
 *     this plan into host memory: 0 = analysis Fourier cube after the gamma
 *     step, complex [N][Lj (m >= 0)][Lj (m' >= 0)]; 1 = after the beta step,
 *     complex [N][2L (beta_b)][Lj (m)] (an S2DW_MW analysis fills its
 *     leading [N][L][Lj]); *nbytes gets the size; host may be NULL to query
 *     only.  Scale j = J+1 is the scaling part (N = 1).
 */
int s2dw_scale_support(s2dw_plan_t plan, int j, int* lo, int* hi);
int s2dw_delta_slab(s2dw_plan_t plan, int l, double* host_out);
int s2dw_stage(s2dw_plan_t plan, int stage, int j, void* host_out, int64_t* nbytes);

/*
 * Stage timing (instrumentation; the paper has no counterpart).
 *   s2dw_profile(plan, 1) resets the counters and makes the next (up to 256)
 *   s2dw_analysis / s2dw_synthesis calls on this plan record CUDA events
 *   around each of their launches, on the call's stream; 0 stops recording.
 *   s2dw_profile_read(plan, ms, ncalls) waits for the recorded calls and
 *   fills ms[13] with per-launch durations (ms) summed over them:
 *   [0] analysis contraction + gamma step, [1] scaling contraction,
 *   [2] beta step, [3] alpha step, chirp-z of the full-band scales,
 *   [4] alpha step, segmented chirp-z of the mid-band scales, [5] alpha
 *   step, direct sums of the small-band scales; [6] synthesis alpha step
 *   (direct sums), [7] alpha step (full-band chirp-z), [8] alpha step
 *   (segmented chirp-z), [9] beta step, [10] contraction, [11] scaling
 *   contraction, [12] final reduction (an empty launch reads 0);
 *   ncalls[2] (may be NULL) gets the numbers of analysis and synthesis calls.
 */
int s2dw_profile(s2dw_plan_t plan, int enable);
int s2dw_profile_read(s2dw_plan_t plan, double* ms, int* ncalls);

/*
 * Launch methods and the autotuner (the paper has no counterpart: these pick
 * among exact evaluations of the same sums, so results agree to rounding).
 *   Choices of a plan, int[3 + 2 (J+2)]:
 *   [0] beta sums of the analysis, [1] beta sums of the synthesis:
 *       0 = one FFT of length 4L per column, 1 = one complex DCT/DST of length
 *       2L per column on the grids where it measured faster (L >= 128 in the
 *       analysis, 128 <= L <= 1024 in the synthesis), the FFT on the others
 *       (both where L is a power of two; a grid with other L keeps its
 *       chirp-z; the DCT/DST is launched once per transform length);
 *       default 1;
 *   [2 + 2j] alpha sums of the analysis of scale j (j = J+1: scaling part),
 *   [3 + 2j] of the synthesis: 0 = direct sums (L_j <= 32), 1 = chirp-z of
 *       the grid's length, 2 = segmented chirp-z (where the plan built its
 *       tables, s2dw_alpha_method);
 *   [last] the contraction's CTA shape (FP32 plans): 0 = both tiles of a
 *       pair of 32-wide blocks per CTA (N <= 5), 1 = one tile per CTA (the
 *       only shape for N > 5), 2 = one tile per CTA at two CTAs per SM
 *       (N <= 5); FP64 plans: 0.
 *   s2dw_plan_choices(plan, choices, n): *n in = capacity, out = entries;
 *     choices == NULL only queries *n; S2DW_EINVAL if the capacity is short.
 *   s2dw_plan_set_choices(plan, choices, n): n must be the plan's count and
 *     every value available (else S2DW_EINVAL); waits for the plan's previous
 *     calls, then rebuilds its launch lists (batched launch lists holding the
 *     plan are dropped).
 *   s2dw_plan_tune(plan, reps, choices, n): times the candidates on the
 *     plan's private stream with scratch buffers it allocates and frees (a
 *     pseudo-random f_lm and the W its analysis writes; coordinate descent:
 *     each direction's beta method, then each scale's alpha method, largest
 *     band first, then the contraction's CTA shape (both directions' times),
 *     the minimum of `reps` round trips per trial, a candidate
 *     kept when it is 3% faster in two measurements with the incumbent
 *     re-timed between them), applies the best and writes it to choices (may
 *     be NULL).  Synchronous; 1 <= reps <= 64.
 */
int s2dw_plan_choices(s2dw_plan_t plan, int* choices, int* n);
int s2dw_plan_set_choices(s2dw_plan_t plan, const int* choices, int n);
int s2dw_plan_tune(s2dw_plan_t plan, int reps, int* choices, int* n);

/*
 * s2dw_delta_table_noalloc: build the Wigner Delta table without allocating.
 *   The paper has no counterpart to this entry point.  It serves callers
 *   that cannot let this library call cudaMalloc: code whose device memory
 *   is owned by another allocator (a framework's caching pool, or a fixed
 *   arena reserved at start-up), or code running where a new allocation
 *   would synchronise the device or is not allowed at all.  Such a caller
 *   allocates the output itself; the only other device memory used is one
 *   fixed 6.3 MB scratch array inside this library, which every GPU that
 *   loads the library keeps until the process exits.  No cudaMalloc,
 *   cudaFree or other allocating call is made.
 *   Lmax: the table covers 0 <= l < Lmax.  1 <= Lmax <= 1024 (the scratch
 *     array's size); Lmax > 1024 returns S2DW_ENOTSUP, Lmax < 1 S2DW_EINVAL.
 *   entries (may be NULL): receives the number of table entries,
 *     32 C (C+1) (C+2) / 3 + (Lmax mod 4) * 8 (C+1) (C+2), C = floor(Lmax/4).
 *   table64: device array of that many doubles (NULL: only report the size,
 *     no device work); table32: NULL or a device array of that many floats
 *     that receives the float32 copy.
 *   Layout (the eighth-domain layout of the plans' FP64 table, without the
 *   zero front pad and read-ahead pad that the plans' copies carry, so this
 *   table is for the caller's own use and cannot stand in for a plan's):
 *     slab l starts at entry
 *     32 C(C+1)(C+2)/3 + (l mod 4) * 8 c(c+1), C = floor(l/4), c = C+1; in it,
 *     Delta^l_{m'm} with m >= 4 floor(m'/4) sits at
 *     16 q c - 8 q (q-1) + 4 r (c-q) + m - 4q, q = floor(m'/4), r = m' mod 4;
 *     the remaining entries follow from Delta_{m'm} = (-1)^{m'-m} Delta_{m m'}
 *     and Delta_{-m',m} = (-1)^{l+m} Delta_{m'm}; padding entries are zero.
 *   Asynchronous on `stream`: the output buffers are cleared and written.
 *   The first call on each device looks up the device address of the scratch
 *   array (cudaGetSymbolAddress) -- make that first call before any stream
 *   capture.  All calls share the one scratch array and its contents stay
 *   from the previous call: calls whose GPU work overlaps (two streams, two
 *   host threads) race and corrupt each other; serialise them.
 */
int s2dw_delta_table_noalloc(int Lmax, double* table64, float* table32, int64_t* entries, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* S2DW_H */
