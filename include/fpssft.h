/*
 * fpssft.h -- C ABI of the FPS-SFT recovery loop on GB300 (sm_103a).
 *
 * FPS-SFT (Wang, Patel, Petropulu, arXiv 1711.11407) recovers the K on-grid D-D complex sinusoids
 * of a cube x(n) = sum_k a_k exp(j 2 pi sum_d k_d n_d / N_d)  (Sec. 2, Eq. sigModel2; D-D in
 * Sec. 2.3) from samples taken along discrete lines.  Every iteration t uses one slope alpha_t
 * and one offset tau_t (both in X_D = [N_0] x ... x [N_{D-1}]) and D+1 lines of length
 * L = LCM(N_0, ..., N_{D-1}) (Lemma 1):
 *     line 0:    s_0(l)     = x([alpha l + tau]_N)                 (Eq. sample_slice)
 *     line d+1:  s_{d+1}(l) = x([alpha l + tau + e_d]_N)           (Sec. 2.3; D+1 lines)
 * their L-point DFTs  s_hat_j(m) = (1/L) sum_l s_j(l) exp(-j 2 pi l m / L)   (Eq. hs),
 * subtracts the bins of the sinusoids recovered so far (construction-subtraction, Sec. 2.2, done
 * on the bins), decodes every 1-sparse bin by the OFDM trick (Eq. decoding) and merges the
 * result into the recovered set.
 *
 * Conventions shared by every call:
 *   - Complex numbers are complex64: two floats (re, im), interleaved.
 *   - A batch holds `batch` cubes with per-signal shapes dims[b][0..D-1] (1 <= D <= 4).  Cubes are
 *     C-order (last dimension fastest) and concatenated in one device buffer; offsets[b] (int64,
 *     device) is the element offset of cube b, which occupies elements [offsets[b], offsets[b] +
 *     N_b) of that buffer.  The library cannot see the buffer's size: offsets outside it are the
 *     caller's error (the Python binding checks them against the tensor before every call).
 *   - L_b = LCM of signal b's dims; L_max = max_b L_b.  Bin and line arrays are
 *     [batch][n_sched][D+1][L_max] complex64; entries m >= L_b of a line are written as zero.
 *   - Schedules alpha, tau are int32 [batch][n_sched][D] (device) with 0 <= alpha_d, tau_d < N_d.
 *     fpssft_recover reads [batch][T_max][D], where T_max is reported by fpssft_plan_get_info.
 *   - Recovered sets are k: int32 [batch][k_cap][D] (frequency indices), a: complex64
 *     [batch][k_cap], count: int32 [batch].
 *   - Device pointers are plain CUDA device addresses; `stream` is a cudaStream_t (NULL = legacy
 *     default stream).  All calls except plan creation/destruction and fpssft_recover_host are
 *     asynchronous on `stream`; they allocate nothing and synchronise nothing, so they can be
 *     recorded into a CUDA graph.
 *   - Ownership: the caller owns every buffer it passes.  The plan owns its own device workspace
 *     (shape table, twiddle tables, work queue, host staging buffers) and frees it in
 *     fpssft_plan_destroy.
 *   - Errors: the return code reports argument validation and launch errors; the message of the
 *     last failure on the calling thread is returned by fpssft_last_error.  Errors found on the
 *     device (recovered-set capacity) are written per signal to out_status after the stream
 *     completes.  No call traps or aborts on the device.
 */
#ifndef FPSSFT_H
#define FPSSFT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  FPSSFT_OK = 0,
  FPSSFT_ERR_INVALID = 1,      /* bad argument: null pointer, dims out of range, bad mode */
  FPSSFT_ERR_CUDA = 2,         /* a CUDA runtime call failed (message names it) */
  FPSSFT_ERR_ALLOC = 3,        /* the plan could not allocate its workspace */
  FPSSFT_ERR_CAPACITY = 4,     /* per signal, in out_status: the recovered set reached k_cap */
  FPSSFT_ERR_TIMEOUT = 5,      /* reserved for bounded device waits (none exist today) */
  FPSSFT_ERR_UNSUPPORTED = 6   /* valid but not implemented: L too long for shared memory, ... */
} fpssft_status;

/* Recovery parameters.  The thresholds implement the 1-sparsity test the paper leaves open
 * (Sec. 2.2 only states that a non-zero bin is 1-sparse with high probability; Sec. 2.1 tests
 * 1-sparsity by equal magnitudes).  For every bin m, with s_j = s_hat_j(m):
 *   T0  |s_0| > theta0;
 *   T1  | |s_{d+1}| - |s_0| | <= rho |s_0| for every d;
 *   T2  |u_d - floor(u_d + 1/2)| <= eta, u_d = N_d phi(s_{d+1} conj(s_0)) / (2 pi), phi in (-pi, pi];
 *   T3  [sum_d (L/N_d) alpha_d k_d]_L = m  with k_d = [floor(u_d + 1/2)]_{N_d}  (Eq. orthogonality);
 * a bin passing all four yields (k, a = s_0 exp(-j 2 pi sum_d k_d tau_d / N_d)) (Eq. decoding). */
typedef struct {
  int T;             /* iterations; 0 = per signal floor(N / ((D+1) L)), the budget of Sec. 3 */
  int k_cap;         /* capacity of each signal's recovered set (>= 1) */
  float theta0;      /* T0 threshold (absolute) */
  float rho;         /* T1 relative magnitude tolerance */
  float eta;         /* T2 distance of the decoded phase from the frequency grid */
  int early_stop;    /* 0: every signal runs its T iterations; 1 (any nonzero value but 2): stop a
                        signal after an iteration in which no bin of line 0 passes T0 after
                        peeling; 2: also stop it after an iteration in which every line-0 bin
                        passing T0 was decoded (what was left on its lines is now recovered) --
                        one iteration earlier on noiseless data (readings of the stop rule: the
                        paper runs T iterations, Sec. 2.2, and counts the samples to perfect
                        recovery, Sec. 3) */
  int peel_mode;     /* 0 = subtract the recovered set's projections from the bins (only mode) */
  int threads;       /* CTA size of the shared-memory-FFT recovery kernel (multiple of 32, <= 1024);
                        0 = library default */
  int ctas_per_sm;   /* resident CTAs per SM for the persistent recovery grid; 0 = occupancy */
  int fp64_decisions;/* nonzero: evaluate T0..T2 in FP64 for every bin.  0 (default): evaluate in
                        FP32 and re-evaluate in FP64 only the bins whose FP32 value falls inside a
                        guard band around a threshold -- the verdicts are the same either way */
  int gather_mode;   /* line-sample loads of fpssft_recover: 0 = library choice (synchronous
                        through L1, except mode 3 on path 3 for L_max < 2048 and on the register-FFT
                        path for batches its mode-3 kernel holds resident at once, and mode 4 on the
                        register-FFT path for larger batches), 1 = synchronous through L1,
                        2 = synchronous cached in L2 only, 3 = asynchronous copies (cp.async) of the
                        next iteration's lines into a shared-memory buffer while the current one
                        computes.  On the register-FFT path modes 1 and 2 prefetch the next
                        iteration into registers instead; 4 = synchronous through L1 with no
                        prefetch (register-FFT path; elsewhere the same as 1); 5 = as 4, with the
                        next iteration's samples hinted into L2 (prefetch.global.L2) right after the
                        FFT (register-FFT path; elsewhere the same as 1) */
  int fft_path;      /* fpssft_recover's kernel: 0 = library choice, 1 = one CTA per signal with the
                        shared-memory mixed-radix FFT (any L), 2 = one warp per line with a register
                        FFT (every L of the batch in {32, 64, 128, 256}), 3 = one CTA per line, the
                        D+1 CTAs of a signal forming a thread-block cluster that exchanges bins
                        through distributed shared memory (`threads` sets the CTA size).  0 picks
                        2 when it applies, else 3 when L_max >= 1024, batch <= 2 x SM count and
                        one line plus the set fit one CTA's shared memory, else 1 */
  int amp_average;   /* 0: amplitude from line tau only (Eq. decoding); nonzero: the mean over the
                        D+1 lines of s_j times the conjugate of line j's offset phase (noisy data) */
  int radix_plan;    /* order of the mixed-radix stages of the shared-memory FFT (paths 1 and 3; the
                        result is the same DFT, only the stage sequence changes):
                        0 = radix 8 as often as possible, then 4, 2, then 3, 5 and larger primes;
                        1 = radix 4 first (then one 2), then the odd factors;
                        2 = the odd factors (3, 5, larger primes) first, then 8, 4, 2;
                        3 = the power of two as radix 8 and 4 stages only (no radix-2 stage unless
                            L's power of two is 2), then the odd factors */
  int host_cubes;    /* fpssft_recover_host only: 0 = copy every cube to the device before the
                        recovery; 1 = when `cubes` is pinned host memory the device can address
                        (cudaHostAlloc, cudaMallocHost or cudaHostRegister), read the samples the
                        gather needs in place over the host link (NVLink-C2C on GB300) and copy only
                        offsets, schedules and results -- FPS-SFT reads a fraction of each cube, so
                        this moves far fewer bytes when the early stop comes soon; other host memory
                        is copied as with 0 */
  int cluster_set;   /* where path 3 keeps each signal's recovered set (list and index): 0 (library
                        choice) or 1 = shared memory when it fits, else plan-owned global workspace;
                        2 = global workspace (L2-resident) always.  Without the set a CTA needs about
                        a third of the shared memory, so smaller CTAs (`threads`) can share an SM and
                        a batch with more clusters than SMs is resident at once -- faster for long
                        runs with small sets (64 noisy 1024^2 images, 256-thread CTAs), slower for
                        short runs with large sets (noiseless images), hence an autotuner candidate
                        rather than the default.  The results do not depend on it */
} fpssft_params;

typedef struct fpssft_plan_s* fpssft_plan_t;

typedef struct {
  int D;
  int batch;
  int L_max;          /* longest line length in the batch */
  int T_max;          /* schedule rows fpssft_recover reads per signal */
  int k_cap;
  int hash_cap;       /* open-addressing table size per signal (power of two >= 2 k_cap) */
  int n_shapes;       /* distinct shapes in the batch */
  int threads;        /* CTA size used by fpssft_recover */
  int grid;           /* persistent CTAs launched by fpssft_recover */
  int smem_bytes;     /* dynamic shared memory per recovery CTA */
  int twiddles_in_smem;
  int prefetch;       /* 1: the next iteration's lines are gathered while the current one computes */
  int fft_path;       /* 1: shared-memory FFT, one CTA per signal; 2: register FFT, one warp per line;
                         3: one CTA per line, a cluster of D+1 CTAs per signal (grid = batch (D+1)) */
  int global_workspace; /* 1: data too large for shared memory lives in plan-owned global
                        workspace (fpssft_recover only): on path 1 the lines and the recovered set
                        (one slice per persistent CTA), on path 3 the recovered set (one slice per
                        signal, 12 bytes per set entry + 8 bytes per index slot) */
} fpssft_plan_info;

/* Create a plan for `batch` signals of dimension D with shapes dims (HOST int64 [batch][D],
 * each N_d >= 1).  Computes L_b = LCM(dims[b]) (Lemma 1), the mixed-radix FFT factorisation of
 * every distinct L, FP64-derived twiddle tables, the per-signal iteration budget and a
 * longest-first work order, and uploads them to device workspace owned by the plan.
 * When the D+1 lines or the recovered set do not fit one CTA's shared memory, fpssft_recover keeps
 * them in plan-owned global workspace (2 x SM count slices on path 1; on path 3 only the set, one
 * slice per signal); fpssft_project, fpssft_lines, fpssft_synth and fpssft_adjoint return
 * FPSSFT_ERR_UNSUPPORTED for a plan whose D+1 lines exceed shared memory.
 * Must be called with the target device current. */
fpssft_status fpssft_plan_create(fpssft_plan_t* out, int D, int batch, const int64_t* dims,
                                 const fpssft_params* params);

/* Same as fpssft_plan_create (the name used by the paper-level description of this interface). */
fpssft_status fpssft_plan(fpssft_plan_t* out, int D, int batch, const int64_t* dims,
                          const fpssft_params* params);

void fpssft_plan_destroy(fpssft_plan_t plan);

fpssft_status fpssft_plan_get_info(fpssft_plan_t plan, fpssft_plan_info* info);

/* Per-signal line length L_b and iteration budget T_b, written to HOST int32 arrays [batch]
 * (either may be NULL). */
fpssft_status fpssft_plan_get_lengths(fpssft_plan_t plan, int32_t* L_out, int32_t* T_out);

/* Line projection (Eq. sample_slice + Eq. hs): for every signal b and schedule row s, the D+1
 * line DFTs s_hat_j(m), written to bins [batch][n_sched][D+1][L_max] (complex64, device).  By the
 * projection-slice identity (Eq. freqSum, Lemma 1) bin m of line j equals the sum, over the
 * frequencies k with [sum_d (L/N_d) alpha_d k_d]_L = m, of the D-D DFT value at k times
 * exp(j 2 pi sum_d k_d (tau_d + [j = d+1]) / N_d). */
fpssft_status fpssft_project(fpssft_plan_t plan, const void* cubes, const int64_t* offsets,
                             const int32_t* alpha, const int32_t* tau, int n_sched, void* bins,
                             void* stream);

/* Raw line samples s_j(l) (Eq. sample_slice, no DFT), same layout as fpssft_project's bins. */
fpssft_status fpssft_lines(fpssft_plan_t plan, const void* cubes, const int64_t* offsets,
                           const int32_t* alpha, const int32_t* tau, int n_sched, void* lines,
                           void* stream);

/* The full recovery loop (Sec. 2.2): for every signal, up to T_b iterations of gather, L-point
 * DFT, subtraction of the recovered set's bins, 1-sparse classification + OFDM decode, merge.
 * One persistent launch processes the whole batch (longest signals first).
 *   alpha, tau:  int32 [batch][T_max][D] (device).
 *   init_count:  NULL, or int32 [batch] (device): resume from the first init_count[b] entries
 *                already present in out_k / out_a (checkpoint / teacher forcing).  The entries
 *                must have distinct frequencies, as fpssft_recover writes them; with repeated
 *                frequencies the resumed set is unspecified (no access leaves the buffers).
 *   out_k, out_a, out_count: the recovered set, entries with |a| <= theta0 dropped, sorted by
 *                row-major linear frequency index.
 *   out_iters:   iterations whose lines were sampled.
 *   out_status:  FPSSFT_OK or FPSSFT_ERR_CAPACITY per signal.
 * Allocates nothing; the caller's buffers and the plan's workspace are the only memory used.  One
 * kernel launch and nothing else is enqueued: the plan's work counter is zero when the plan is
 * created and every launch returns it to zero, so launches of one plan must be ordered (one stream,
 * or events between streams).
 * `cubes` may also point to pinned (page-locked, mapped) host memory: the gather then reads the
 * samples it needs over the host link (on GB300 the cache-coherent NVLink-C2C) instead of the
 * caller copying every cube to the device first. */
fpssft_status fpssft_recover(fpssft_plan_t plan, const void* cubes, const int64_t* offsets,
                             const int32_t* alpha, const int32_t* tau, const int32_t* init_count,
                             int32_t* out_k, void* out_a, int32_t* out_count, int32_t* out_iters,
                             int32_t* out_status, void* stream);

/* fpssft_recover on HOST buffers: cubes (complex64, total elements = sum N_b), offsets, alpha,
 * tau and init_count in host memory (pinned memory gives full copy bandwidth).  The call copies
 * the inputs into plan-owned device staging (allocated on the first call that needs it; with
 * fpssft_params.host_cubes = 1 pinned cubes are read in place instead of copied), runs the
 * recovery on `stream`, copies every output back into the host arrays and synchronises the stream
 * before returning. */
fpssft_status fpssft_recover_host(fpssft_plan_t plan, const void* cubes, const int64_t* offsets,
                                  const int32_t* alpha, const int32_t* tau, const int32_t* init_count,
                                  int32_t* out_k, void* out_a, int32_t* out_count, int32_t* out_iters,
                                  int32_t* out_status, void* stream);

/* Sparse synthesis (Eq. freqSum applied to a set {(k_i, a_i)}, the construction step of Sec. 2.2):
 *   bins[b][s][j][m] = sum over i < count[b] with [sum_d (L/N_d) alpha_d k_{i,d}]_L = m of
 *                      a_i exp(j 2 pi sum_d k_{i,d} (tau_d + [j = d+1]) / N_d).
 * accumulate = 0 overwrites bins, +1 adds to them, -1 subtracts from them (the peel). */
fpssft_status fpssft_synth(fpssft_plan_t plan, const int32_t* alpha, const int32_t* tau,
                           int n_sched, const int32_t* k, const void* a, const int32_t* count,
                           int accumulate, void* bins, void* stream);

/* One iteration's classification, decode and merge on precomputed bins [batch][1][D+1][L_max]
 * (already peeled), updating the set (k, a, count) in place, as in fpssft_recover.  Writes the
 * number of line-0 bins passing T0 to t0_count [batch], the number of bins decoded (T0..T3
 * passed) to accepted [batch] (nullable; the two are equal when the decoded-stop of early_stop = 2
 * applies) and ORs FPSSFT_ERR_CAPACITY into status.
 * Building block of the unfused, per-iteration host-driven form of the loop.  Returns
 * FPSSFT_ERR_UNSUPPORTED (nothing launched) when one signal's set (k_cap entries and index) does
 * not fit one CTA's shared memory. */
fpssft_status fpssft_decode(fpssft_plan_t plan, const void* bins, const int32_t* alpha,
                            const int32_t* tau, int32_t* k, void* a, int32_t* count,
                            int32_t* t0_count, int32_t* accepted, int32_t* status, void* stream);

/* Drop entries with |a| <= theta0 and sort each signal's set by linear index (in place).
 * FPSSFT_ERR_UNSUPPORTED as for fpssft_decode. */
fpssft_status fpssft_finalize(fpssft_plan_t plan, int32_t* k, void* a, int32_t* count, void* stream);

typedef enum { FPSSFT_ADJ_PROJECT = 0, FPSSFT_ADJ_SYNTH = 1 } fpssft_adj_mode;

/* Adjoints (conjugate transposes) of the two linear maps above.
 *   FPSSFT_ADJ_PROJECT: grad_out (cube layout at `offsets`, complex64) += P^H grad_bins, i.e. for
 *     every line the inverse-direction DFT scaled by 1/L,  (1/L) sum_m g_j(m) exp(+j 2 pi l m / L),
 *     scatter-added at the line's grid points (atomic; lines may revisit a point).  k, count
 *     unused.
 *   FPSSFT_ADJ_SYNTH: grad_out [batch][k_cap] complex64 (overwritten for i < count[b]) =
 *     sum over schedule rows and lines of conj(exp(j 2 pi sum_d k_{i,d}(tau_d + [j = d+1]) / N_d))
 *     g_j(m(k_i)).  offsets unused.
 * grad_bins: [batch][n_sched][D+1][L_max] complex64. */
fpssft_status fpssft_adjoint(fpssft_plan_t plan, fpssft_adj_mode mode, const void* grad_bins,
                             const int64_t* offsets, const int32_t* alpha, const int32_t* tau,
                             int n_sched, const int32_t* k, const int32_t* count, void* grad_out,
                             void* stream);

/* Least-squares amplitude refinement on a fixed support.  The decode (Sec. 2.2, Eq. decoding)
 * reads each amplitude from one bin of one line; over n_sched schedule rows every line carries
 * the same amplitudes (Eq. freqSum), y_r = S_r a + noise, with y_r the D+1 line DFTs of row r
 * (Eq. sample_slice, Eq. hs) and S_r the synthesis of fpssft_synth.  This call solves, per signal,
 *     min_a  sum_r || y_r - S_r a ||^2
 * by conjugate gradients on the normal equations (S^H S) a = S^H y (the least-squares step is an
 * addition of this library; the paper stops at the decode).  Everything runs on the device, two
 * launches per iteration and none of them waits on the host; signals whose normal-equation
 * residual falls below tol^2 of its start stop changing (later iterations leave them as they are).
 *   bins:      device complex64 [batch][n_sched][D+1][L_max], y = fpssft_project of the cubes on the
 *              same rows;
 *   alpha, tau: device int32 [batch][n_sched][D], the rows;
 *   k, count:  device, the support (entries i < count[b] of k [batch][k_cap][D]; entries off the
 *              grid are ignored);
 *   a:         device complex64 [batch][k_cap]: the starting amplitudes on entry, the refined ones on
 *              return (entries i >= count[b] untouched);
 *   iters:     conjugate-gradient iterations (0: only the residual);
 *   workspace: device, at least fpssft_refine_workspace_size bytes, 256-byte aligned, owned by the
 *              caller (contents need no initialisation; overwritten);
 *   resid:     nullable device float [batch]: || y - S a || over all rows after the last iteration.
 * Arithmetic: FP32 vectors and bins, FP64 CG scalars.  FPSSFT_ERR_UNSUPPORTED when the D+1 lines
 * of one row do not fit one CTA's shared memory. */
fpssft_status fpssft_refine_workspace_size(fpssft_plan_t plan, size_t* bytes);
fpssft_status fpssft_refine(fpssft_plan_t plan, const void* bins, const int32_t* alpha, const int32_t* tau,
                            int n_sched, const int32_t* k, const int32_t* count, void* a, int iters,
                            float tol, void* workspace, size_t workspace_bytes, float* resid,
                            void* stream);

/* Size of the fixed device scratch used by fpssft_recover_noalloc (bytes). */
#define FPSSFT_NOALLOC_SCRATCH_BYTES (1 << 20)

/* fpssft_recover without any device allocation (no counterpart in the paper: this is about how
 * the library obtains memory, not about the method).  For callers that cannot allocate device
 * memory when they recover -- code that runs under a memory pool or arena owned by someone else,
 * inside regions where cudaMalloc is forbidden or would synchronise, or within a fixed memory
 * budget.  No plan is needed: the tables a plan would allocate (shapes, per-signal iteration
 * budgets, work order, twiddles) and the work counter are placed in one file-scope device array
 * of FPSSFT_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds until the process
 * exits.  The call allocates nothing on the device and calls no allocating CUDA or library routine.
 *   D, batch, dims (HOST int64 [batch][D]), params: as for fpssft_plan_create.
 *   cubes, offsets, alpha, tau, init_count, out_*: as for fpssft_recover, on the device; alpha and
 *     tau are [batch][T_max][D] with T_max = params->T when T > 0, else the largest per-signal
 *     budget floor(N_b / ((D+1) L_b)).
 * Limits: the tables must fit the array -- about 12 bytes per signal plus one 8-byte twiddle per
 * line position of every distinct line length, and at most 64 distinct shapes.  The call always
 * runs the one-CTA-per-signal kernel with the D+1 lines, their FFT partner and the recovered set
 * in shared memory, so 16 (D+1) L_max + (12 + 4 D) k_cap + 8 H bytes (H the power of two >= 2 k_cap;
 * plus the twiddles when they fit) must stay within one CTA's 227 KB; the plan-based
 * fpssft_recover has global-memory variants for larger lines or sets, this call has none.
 * Requests beyond either limit return FPSSFT_ERR_UNSUPPORTED with a message and launch nothing.
 * The first call on a device also looks up the array's device address and raises the recovery
 * kernel's shared-memory limit; make that first call before any stream capture.  The tables reach
 * the array inside the parameters of small copy kernels launched on `stream` before the recovery
 * (one per 32 000 bytes; the first also clears the work counter), so the call reads no host memory
 * after it returns and does not wait for work already queued on `stream`.
 * Every call shares the one array and it keeps the last call's contents, so calls whose work
 * overlaps on the GPU (different streams, or different host threads) race: issue them one after
 * another on one stream. */
fpssft_status fpssft_recover_noalloc(int D, int batch, const int64_t* dims, const fpssft_params* params,
                                     const void* cubes, const int64_t* offsets, const int32_t* alpha,
                                     const int32_t* tau, const int32_t* init_count, int32_t* out_k,
                                     void* out_a, int32_t* out_count, int32_t* out_iters,
                                     int32_t* out_status, void* stream);

/* Measurement helper (no counterpart in the paper): the random-gather ceiling the line gather is
 * compared against.  threads_total threads each read reads_per_thread 8-byte elements at
 * pseudo-random positions of buf (device, n_elems complex64 elements, a power of two; use a
 * buffer much larger than L2), plus the following element when pair = 1, and write one complex64
 * per thread to out (device, threads_total elements).  load_mode 0 loads through L1
 * (ld.global.nc), 1 caches in L2 only (ld.global.cg).  Asynchronous on stream. */
fpssft_status fpssft_probe_gather(const void* buf, int64_t n_elems, int reads_per_thread, int threads_total,
                                  int load_mode, int pair, void* out, void* stream);

/* The line gather reads isolated 8-byte samples; by default the memory system may fetch a whole
 * 128-byte line from DRAM for each.  This sets the current device's L2 fetch-granularity hint
 * (cudaLimitMaxL2FetchGranularity: 0, 32, 64 or 128 bytes) for the calling process's context --
 * it affects every kernel of the process and nothing outside it -- and returns the previous value
 * in *previous (nullable).  bytes < 0 only queries. */
fpssft_status fpssft_l2_fetch_granularity(int bytes, int* previous);

/* Tracing (no counterpart in the paper).  A library built with -DFPSSFT_PHASE_TIMERS (the Python
 * package's `phases` module builds it as libfpssft_phases.so) times the phases of the three
 * recovery kernels with the SM cycle counter: thread 0 of every CTA adds up the cycles between CTA
 * barriers placed at the phase boundaries and, when the CTA ends, adds them to one device array.
 * fpssft_phase_read waits for the device, copies that array into out (host, FPSSFT_PHASE_WORDS
 * values) and clears it:
 *   out[0 .. FPSSFT_PHASE_COUNT-1]  cycles per phase summed over CTAs, in the order setup,
 *                                   gather, FFT, peel, decode (classify and merge), exchange (the
 *                                   cluster barriers; cluster path only), output;
 *   out[FPSSFT_PHASE_COUNT]         CTAs that contributed (each CTA of each launch once);
 *   out[FPSSFT_PHASE_COUNT + 1]     recovery iterations those CTAs ran;
 *   out[FPSSFT_PHASE_COUNT + 2]     their cycles from start to end of the kernel;
 *   out[FPSSFT_PHASE_COUNT + 3]     the global-timer nanoseconds of the same spans.
 * The barriers make a timed launch slower than a plain one; its results are the same.  The default
 * build returns FPSSFT_ERR_UNSUPPORTED and touches nothing. */
#define FPSSFT_PHASE_COUNT 7
#define FPSSFT_PHASE_WORDS (FPSSFT_PHASE_COUNT + 4)
fpssft_status fpssft_phase_read(int64_t* out);

/* Host-only helper (no device work): the radix of each stage of the L-point mixed-radix FFT under
 * radix plan `radix_plan` (fpssft_params.radix_plan), in the order the stages run.  radices: host,
 * room for 24 entries; *n_stages receives their number.  The stages multiply to L (the L-point DFT
 * of Eq. hs factored Cooley-Tukey style); FPSSFT_ERR_INVALID for L outside [1, 2^24] or an unknown
 * plan, FPSSFT_ERR_UNSUPPORTED beyond 24 stages. */
fpssft_status fpssft_fft_stages(int L, int radix_plan, int32_t* radices, int32_t* n_stages);

/* Message of the last failed call on this thread ("" when none). */
const char* fpssft_last_error(void);

/* Library version string. */
const char* fpssft_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FPSSFT_H */
