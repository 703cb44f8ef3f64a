/*
 * fastmnmf.h — C ABI of libfastmnmf.so, a GB300 (sm_103a) implementation of FastMNMF:
 * Sekiguchi, Nugraha, Bando, Yoshii, "Fast Multichannel Source Separation Based on
 * Jointly Diagonalizable Spatial Covariance Matrices", EUSIPCO 2019 (arXiv 1903.03237).
 *
 * Problem (Sec. II-A-1, Eqs. 1-2; Sec. III-A-1, Eq. 16): an observed multichannel STFT
 * X in C^{F x T x M} is a sum of N source images x_ftn ~ CN(0, lambda_ftn G_nf) whose
 * spatial covariances are jointly diagonalised per bin, Q_f G_nf Q_f^H = Diag(g~_nf),
 * with NMF source PSDs lambda_ftn = sum_k w_nkf h_nkt (Sec. II-B-2, Eq. 9).  The library
 * estimates W, H, g~ and Q by the convergence-guaranteed MM + iterative-projection
 * algorithm of Sec. III (Eqs. 17-24) and separates the sources with the multichannel
 * Wiener filter of Eq. 3.
 *
 * Conventions for every call:
 *  - Layouts are row-major, last index fastest.  Complex numbers are (re, im) pairs of
 *    the stated real type, interleaved.
 *      X    complex64  [F][T][M]          observed mixture
 *      W    float32    [N][K][F]          NMF bases        w_nkf >= 0
 *      H    float32    [N][K][T]          NMF activations  h_nkt >= 0
 *      G    float32    [N][F][M]          diagonal SCMs    g~_nfm >= 0
 *      Q    complex64  [F][M][M]          diagonalisers; row m of Q_f is q_fm^H (Eq. 16)
 *      out  complex64  [N][F][T][M]       separated source images (all M channels)
 *  - Pointers marked "host" are ordinary host memory; "device" pointers are CUDA device
 *    memory of the current device and must be 16-byte aligned.  Device inputs are read on
 *    the context stream: the caller must have completed (or ordered before that stream)
 *    whatever work produces them; device outputs are ready once the context stream has
 *    passed the call.
 *  - Ownership: the caller owns every buffer it passes; the library copies what it
 *    needs during the call (device->device for device inputs) and never keeps a caller
 *    pointer.  The context owns all device state until fmnmf_destroy.
 *  - Errors: every call returns an fmnmf_status and never aborts.  Argument errors
 *    (FMNMF_EINVAL) change no state.  Errors found on the device (non-finite values, a
 *    singular IP system) are recorded in a device status word, reported by the next
 *    synchronising call (fmnmf_sync, fmnmf_loglik, fmnmf_get_state, fmnmf_separate) and
 *    stay sticky until fmnmf_set_state or fmnmf_reset.  fmnmf_last_error gives a
 *    message.
 *  - Threads: a context is used by one host thread at a time; separate contexts are
 *    independent.  All device work is ordered on the context's stream.
 */
#ifndef FASTMNMF_H
#define FASTMNMF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmnmf_ctx fmnmf_ctx;

typedef enum {
  FMNMF_OK = 0,
  FMNMF_EINVAL = 1,      /* bad argument (shape, pointer, option)                  */
  FMNMF_ENOMEM = 2,      /* device allocation failed or over the HBM budget         */
  FMNMF_ECUDA = 3,       /* a CUDA runtime call failed                              */
  FMNMF_ENONFINITE = 4,  /* NaN/Inf in the input or produced by an update           */
  FMNMF_ESINGULAR = 5,   /* an IP system (Q_f V_fm) had a vanishing pivot            */
  FMNMF_ETIMEOUT = 6,    /* a bounded device wait expired                           */
  FMNMF_EBUSY = 7        /* resource (server slot) not available now                */
} fmnmf_status;

/* Blocks of the update (Sec. III): W (Eq. 23), H (Eq. 24), g~ (Eq. 21), Q (Eqs. 18-20). */
enum { FMNMF_UPDATE_W = 1, FMNMF_UPDATE_H = 2, FMNMF_UPDATE_G = 4, FMNMF_UPDATE_Q = 8,
       FMNMF_UPDATE_ALL = 15 };

/* Arithmetic of the contractions.  FP32: every sum in float32 on CUDA cores.  BF16 / TF32:
 * the NMF and SCM contractions on the tensor cores with float32 accumulation; BF16 splits
 * every operand into BF16 hi and lo parts and takes each product as hi*hi + hi*lo + lo*hi
 * (about 16 significant bits per operand), TF32 rounds the NMF operands to TF32 (11 bits) and
 * splits the SCM operands like BF16.  In every form
 * the M x M IP solves (Eqs. 19-20), their normalisation and log|det Q_f|^2 run in float-float
 * arithmetic (an unevaluated sum of two float32 values, about 48 significand bits) on the
 * FP32 pipes, not in float64: GB300's float64 rate is a small fraction of its float32 rate.
 * Only the per-bin preparation of a newly set Q (its inverse and log-determinant) uses
 * float64.  The per-sum operations and their error bounds are those of the error-free
 * transformations (TwoSum, TwoProduct by FMA) and of one Newton step for the reciprocal and
 * the reciprocal square root; the log-determinant adds log(s) of the row updates with log(hi)
 * correct to float32 rounding plus the first-order lo/hi term. */
enum { FMNMF_PREC_FP32 = 0, FMNMF_PREC_BF16 = 1, FMNMF_PREC_TF32 = 2 };

/* Launch schedule of the FP32 form.
 *  SWEEP: one tiled launch per block of the iteration (W, H, g~, V_fm, the IP with x~; x~ in a
 *         launch of its own beyond 1024 frames): five or six launches.
 *  FUSED: two launches per iteration.  Every block but the H update (Eq. 24, a sum over bins)
 *         is independent per frequency bin, so one kernel runs, per bin, the g~ update, V_fm
 *         and the IP update, the normalisation, x~, the bin's log-likelihood terms and the W
 *         update of the next iteration; a second kernel runs the H update over tiles of
 *         frames and refreshes lambda.  Needs N*M <= 256 and the bin's tiles (about
 *         4 (N*K + 260 N + 1030 MAXM) bytes, MAXM the channel bucket 2, 4 or 8) within shared memory.
 *  AUTO:  FUSED when it applies, else SWEEP.  The mixed-precision forms ignore the field. */
enum { FMNMF_SCHED_AUTO = 0, FMNMF_SCHED_SWEEP = 1, FMNMF_SCHED_FUSED = 2 };

/* Source model (Sec. III-B).  NMF: lambda_ftn = sum_k w_nkf h_nkt (Eq. 9): FastMNMF (Sec.
 * III-C-2).  FREE: the unconstrained source model, lambda_ftn estimated directly by the
 * multiplicative rule of Eq. 22 (K is ignored): FastFCA (Sec. III-C-1) with the IP update of
 * Q.  FREE runs in the FP32 form with the fused schedule only. */
enum { FMNMF_SOURCE_NMF = 0, FMNMF_SOURCE_FREE = 1 };

typedef struct {
  int precision;          /* FMNMF_PREC_*                                      (default FP32) */
  unsigned update_mask;   /* FMNMF_UPDATE_* bits applied by fmnmf_iterate      (default ALL)  */
  int normalise;          /* 1: scale normalisation (see fmnmf_iterate)       (default 1)    */
  void* stream;           /* cudaStream_t for all device work; NULL = a private stream        */
  size_t hbm_budget;      /* 0 = unlimited; else init fails with ENOMEM above it              */
  int schedule;           /* FMNMF_SCHED_*                                     (default AUTO) */
  int source_model;       /* FMNMF_SOURCE_*                                    (default NMF)  */
} fmnmf_opts;

/* Fills *opts with the defaults above. */
fmnmf_status fmnmf_default_opts(fmnmf_opts* opts);

/*
 * Creates a context for one mixture and sets the initial state.
 *  X           complex64 [F][T][M], host (x_on_device = 0) or device (x_on_device = 1).
 *              Must be finite (checked on the device after the copy; FMNMF_ENONFINITE
 *              otherwise, with the index of the first non-finite float in the message).
 *  F, T        >= 1 bins and frames; M in [1, 8] channels; N >= 1 sources; K >= 1 bases.
 *  seed        initial state (the paper fixes none for FastMNMF; Sec. IV-A only gives
 *              one for its DP experiments):  with u_i the i-th output of the counter-based
 *              SplitMix64 stream of `seed` (output i = mix(seed + (i+1)*0x9E3779B97F4A7C15),
 *              top 53 bits / 2^53), W[n][k][f] = 0.1 + u_{(nK+k)F+f},
 *              H[n][k][t] = 0.1 + u_{NKF+(nK+k)T+t}; g~[n][f][m] = (m == n mod M ? 1 : 0.01)
 *              divided by its sum over m; Q_f = I.
 *  opts        may be NULL (defaults).
 * On success *out receives the context; x~, y~ and the log-likelihood of the initial state
 * are computed.  Device memory: about (8 + 4 + 4) F T M + 4 N K (F + T) bytes + scratch.
 */
fmnmf_status fmnmf_init(fmnmf_ctx** out, const void* X, int x_on_device, int F, int T, int M,
                        int N, int K, uint64_t seed, const fmnmf_opts* opts);

/* Device bytes a context of this shape and options occupies (its arena, plus the Wiener
 * output buffer fmnmf_separate allocates for a host destination).  No device memory is
 * touched; the current device's properties are used for the tiling. */
fmnmf_status fmnmf_footprint(int F, int T, int M, int N, int K, const fmnmf_opts* opts, size_t* bytes);

/* Replaces the mixture of an existing context (same F, T, M) and re-initialises the state
 * from `seed` as fmnmf_init does, reusing the context's device memory.  A non-finite X
 * returns FMNMF_ENONFINITE after it has replaced the mixture: reset again with a finite X
 * before iterating. */
fmnmf_status fmnmf_reset(fmnmf_ctx* ctx, const void* X, int x_on_device, uint64_t seed);

/* Restores the state the context had right after its last fmnmf_init, fmnmf_reset or
 * fmnmf_set_state (device-side copies, asynchronous on the context stream) and clears the
 * error word: the next fmnmf_iterate starts a fresh estimation of the same mixture. */
fmnmf_status fmnmf_restart(fmnmf_ctx* ctx);

/*
 * Runs n_iter >= 0 iterations of FastMNMF (Sec. III-C-2: NMF source model in the jointly
 * diagonalisable spatial model).  One iteration, in this order, each block from the
 * current parameters (so each is an exact MM / IP step and Eq. 17 never decreases):
 *   W  <- W * sqrt(num/den)                                   (Eq. 23)
 *   H  <- H * sqrt(num/den)                                   (Eq. 24)
 *   g~ <- g~ * sqrt(num/den)                                  (Eq. 21)
 *   for m = 1..M:  q_fm <- (Q_f V_fm)^-1 e_m,  q_fm /= sqrt(q^H V_fm q)   (Eqs. 18-20)
 *   x~ <- |Q_f x_ft|^2; scale normalisation (if opts.normalise):
 *     Q_f /= sqrt(tr(Q_f Q_f^H)/M), g~_nf scaled to match; g~_nf /= sum_m g~_nfm with
 *     w_nkf scaled to match; w_nk /= sum_f w_nkf with h_nk scaled to match
 *   (these leave every y~ and the log-likelihood unchanged);
 *   log-likelihood of the new state (Eq. 17).
 * With the unconstrained source model (FastFCA, Sec. III-C-1) the W and H updates are
 * replaced by  lambda_ftn <- lambda_ftn * sqrt(num/den)  (Eq. 22, every point) and the nu
 * normalisation scales lambda_ftn instead of w_nkf (update_mask bit W selects the lambda
 * update, bit H is ignored).  In every form the mu normalisation is applied once at the end
 * of each call, and of each run of at most 100 iterations within it (it commutes with every
 * update, so the state is that of the per-iteration normalisation up to rounding; results
 * therefore depend on how iterations are split into calls, by rounding only), and the
 * log-likelihood is summed for the last iteration only.
 * Asynchronous: enqueued on the context stream; device errors surface at the next
 * synchronising call.
 */
fmnmf_status fmnmf_iterate(fmnmf_ctx* ctx, int n_iter);

/* Waits for the context stream and reports any device-side error. */
fmnmf_status fmnmf_sync(fmnmf_ctx* ctx);

/* Non-blocking: FMNMF_EBUSY while work enqueued on the context stream is still running;
 * otherwise what fmnmf_sync returns (without waiting). */
fmnmf_status fmnmf_query(fmnmf_ctx* ctx);

/* Synchronises and returns the log-likelihood of the current state: Eq. 17 including the
 * constant -F T M log(pi) that the paper's "=c" drops (the true log-density of Eq. 2). */
fmnmf_status fmnmf_loglik(fmnmf_ctx* ctx, double* ll);

/*
 * Multichannel Wiener filter, Eq. 3, in diagonalised form (Eq. 16 substituted):
 *   x_ftn = Q_f^-1 ( (lambda_ftn g~_nf / y~_ft) (elementwise) Q_f x_ft )
 * for every source n and every channel.  out: complex64 [N][F][T][M], host
 * (out_on_device = 0; the call synchronises) or device (asynchronous).
 */
fmnmf_status fmnmf_separate(fmnmf_ctx* ctx, void* out, int out_on_device);

/* Copies the state to host buffers (any may be NULL; W and H must be NULL for the
 * unconstrained source model, whose lambda fmnmf_get_lambda returns).  Synchronises. */
fmnmf_status fmnmf_get_state(fmnmf_ctx* ctx, float* W, float* H, float* G, void* Q);

/* Unconstrained source model (FastFCA) only.  get: copies lambda, float32 [N][F][T] (host),
 * and, if not NULL, g~ and Q; synchronises.  set: sets lambda, g~ and Q (host; all three
 * required, finite, lambda and g~ >= 0, Q_f non-singular), recomputes x~, y~ and the
 * log-likelihood and clears the error word, as fmnmf_set_state does.  The initial state of
 * fmnmf_init for this model: lambda[n][f][t] = 0.1 + u_{(nF + f)T + t} (the SplitMix64
 * uniforms of fmnmf_init), g~ and Q as for the NMF model. */
fmnmf_status fmnmf_get_lambda(fmnmf_ctx* ctx, float* lam, float* G, void* Q);
fmnmf_status fmnmf_set_lambda(fmnmf_ctx* ctx, const float* lam, const float* G, const void* Q);

/* Sets the state from host buffers (all four required, finite, W/H/G >= 0, Q_f
 * non-singular), recomputes x~, y~ and the log-likelihood and clears the error word. */
fmnmf_status fmnmf_set_state(fmnmf_ctx* ctx, const float* W, const float* H, const float* G,
                             const void* Q);

/*
 * Spectral initialisation of g~ and Q (Sec. IV-A): the SCM of source 1 starts as the
 * average observed SCM G_1f = (1/T) sum_t x_ft x_ft^H and the others as the identity; with
 * G_1f = U_f Diag(e_f) U_f^H (eigenvalues in descending order), Q_f = U_f^H diagonalises
 * them all: g~_1f = e_f, g~_nf = 1 for n >= 2.  The nu normalisation of fmnmf_iterate then
 * divides g~_nf by its sum over m and multiplies w_nkf (lambda_ftn for the unconstrained
 * source model) by it; H is kept.  The eigendecomposition runs on the device in float64
 * (cyclic complex Jacobi rotations, one thread per bin); Q_f is unitary up to rounding.
 * Like fmnmf_set_state it recomputes x~, y~ and the log-likelihood, clears the error word
 * and makes this the state fmnmf_restart returns to.  A bin whose average SCM has no
 * positive eigenvalue (no observed power) is reported as FMNMF_ESINGULAR.  Synchronises.
 */
fmnmf_status fmnmf_init_spectral(fmnmf_ctx* ctx);

/*
 * Front end: the STFT that produces X from multichannel signals and its inverse, which
 * turns separated images back into signals (Sec. IV-A: window of L = 1024 points, shift
 * of 256).  The paper names neither window nor framing; here w_j = (1 - cos(2 pi j/L))/2
 * (periodic Hann), frame t covers samples t*hop .. t*hop + L - 1 (zeros past the end),
 *   X[f][t][m] = sum_j w_j x_m[t*hop + j] exp(-2 pi i f j / L),  f = 0 .. L/2 (F = L/2+1),
 * and the number of frames is T = 1 if S <= L, else 1 + ceil((S - L) / hop)
 * (fmnmf_stft_frames).  The inverse takes each frame's inverse real DFT (the imaginary
 * parts of bins 0 and L/2 are ignored), multiplies it by w, overlap-adds the frames and
 * divides every sample by sum_t w_{s - t hop}^2; samples where that sum is below 1e-10 of
 * its largest value are 0.
 *  L     power of two in [16, 4096]; hop in [1, L]; S >= 1 samples.
 *  x     device float32 [M][S] signals (4-byte aligned); X  device complex64 [F][T][M].
 *  Y     device complex64 [B][F][T][M] (B batches of images, e.g. the [N][F][T][M] output
 *        of fmnmf_separate); y device float32 [B][M][S]; (T - 1) * hop + L >= S.
 *  stream  cudaStream_t for the work (NULL = legacy default stream); asynchronous.
 * Computation in float32 (radix-2 FFT in shared memory; twiddles exact-argument sincospi).
 * fmnmf_istft takes B*M*T*L*4 bytes of stream-ordered scratch (cudaMallocAsync) and
 * returns FMNMF_ENOMEM if that fails.  Argument errors return FMNMF_EINVAL and launch
 * nothing (message via fmnmf_last_error(NULL)).
 */
fmnmf_status fmnmf_stft_frames(int S, int L, int hop, int* T);
fmnmf_status fmnmf_stft(const float* x, int M, int S, int L, int hop, void* X, void* stream);
fmnmf_status fmnmf_istft(const void* Y, int B, int F, int T, int M, int S, int L, int hop, float* y,
                         void* stream);

/* Shapes of a context (any pointer may be NULL). */
fmnmf_status fmnmf_shape(const fmnmf_ctx* ctx, int* F, int* T, int* M, int* N, int* K);

/* Frees the context and its device memory.  NULL is accepted. */
fmnmf_status fmnmf_destroy(fmnmf_ctx* ctx);

/* Message for the last error on ctx (or of the calling thread when ctx is NULL). */
const char* fmnmf_last_error(const fmnmf_ctx* ctx);

/*
 * Kernel timing, for measurement only.  kinds is a bit mask of kernel classes (bit i =
 * class i, named by fmnmf_kernel_name(i); -1 = all, 0 = off).  While it is non-zero, every
 * launch of a selected class made by fmnmf_iterate / fmnmf_separate is bracketed by CUDA
 * events on the context stream (inside the captured graphs as event-record nodes).
 * fmnmf_kernel_times synchronises and returns, for each class i < *n, the summed
 * milliseconds and launch count since the last call, then resets them.
 */
fmnmf_status fmnmf_set_timing(fmnmf_ctx* ctx, int kinds);
fmnmf_status fmnmf_kernel_times(fmnmf_ctx* ctx, double* ms, long long* launches, int* n);
const char* fmnmf_kernel_name(int i);

/*
 * Batches: several contexts (independent mixtures, any shapes and precisions) iterated by
 * one CUDA graph launch.  fmnmf_batch_create captures nothing yet; the first
 * fmnmf_batch_iterate for a given chunk length captures every member's iteration into
 * one graph with one branch per context (forked from and joined to the batch's own
 * stream), so the members' kernels overlap on the device; later calls replay it.  Each
 * member computes exactly what fmnmf_iterate would (same kernels, same results).  The
 * contexts must use distinct streams (the default private streams do), stay alive while
 * the batch exists, and not be iterated on their own while a batch call is in flight.
 * fmnmf_batch_sync waits for the batch and reports the first member error.
 */
typedef struct fmnmf_batch fmnmf_batch;
fmnmf_status fmnmf_batch_create(fmnmf_ctx* const* ctxs, int n, fmnmf_batch** out);
fmnmf_status fmnmf_batch_iterate(fmnmf_batch* batch, int n_iter);
fmnmf_status fmnmf_batch_sync(fmnmf_batch* batch);
fmnmf_status fmnmf_batch_destroy(fmnmf_batch* batch);

/*
 * Launch-shape tuning.  Each context plans its launches to fill the GPU alone: the inner
 * split counts of the tiled sweeps (plain form) or of the tensor-core V_fm and g~ kernels
 * and the split-K GEMMs of the W and H sums (mixed form).  The tuner times whole iterations
 * (n_iter per trial, from a saved copy of the state, which is restored afterwards) for
 * those split counts scaled by 1, 3/4, 1/2, 3/8, 1/4, 3/16 and 1/8 and keeps the fastest:
 *  - fmnmf_autotune: coordinate descent over the context's four tunable launches;
 *  - fmnmf_batch_autotune: one scale for every tunable launch of every member, timed on the
 *    whole batch (members running together do better with smaller grids).
 * speedup (may be NULL) receives the first trial's time over the best one.  Fewer splits
 * change the order of the split sums, so results differ from an untuned context by
 * rounding; fmnmf_get_tuning / fmnmf_set_tuning read and set the scales (8 floats in
 * (0, 1]: W, H, g~, y~/V sweeps, V_fm and g~ tensor-core kernels, W and H GEMMs), so that a
 * tuned shape can be reproduced or cached.  Synchronising.
 */
fmnmf_status fmnmf_autotune(fmnmf_ctx* ctx, int n_iter, double* speedup);
fmnmf_status fmnmf_batch_autotune(fmnmf_batch* batch, int n_iter, double* speedup);
fmnmf_status fmnmf_get_tuning(const fmnmf_ctx* ctx, float* scales);
fmnmf_status fmnmf_set_tuning(fmnmf_ctx* ctx, const float* scales);

/*
 * Serving (continuous batching).  A server accepts separation requests of any shape from
 * any thread and returns each one's separated images.  Its scheduler thread:
 *  - admits queued requests in arrival order while fewer than max_active are resident
 *    and their footprint (fmnmf_footprint) fits the HBM budget; the context and state of
 *    an admitted request stay resident on the device until it completes;
 *  - advances every resident request in steps of iters_per_step iterations on its own
 *    stream, so the kernels of resident requests overlap; a request's next step is
 *    enqueued as soon as its previous one has finished (no request waits for another's
 *    step), and new arrivals are admitted between steps;
 *  - separates a request that has run its iterations (Eq. 3) into a host buffer, frees
 *    its device memory and marks it done.
 * A request's results equal those of a context running it alone (fmnmf_init, fmnmf_iterate
 * with iters_per_step iterations per call, fmnmf_separate, the same seed).  Latency =
 * completion - submission.
 *  hbm_budget      device bytes for admitted requests (0 = 70 % of the free memory at
 *                  creation); a request larger than it is rejected with FMNMF_ENOMEM.
 *  max_active      resident requests (0 = 16); iters_per_step (0 = 10); precision FMNMF_PREC_*.
 * submit copies X (host, complex64 [F][T][M]) and returns at once; wait blocks up to
 * timeout_s; result copies the images ([N][F][T][M] complex64, host) and the final
 * log-likelihood and forgets the request (a failed request returns its error).  destroy
 * drops queued requests, finishes the resident ones and frees everything.
 */
typedef struct fmnmf_server fmnmf_server;
enum { FMNMF_JOB_QUEUED = 0, FMNMF_JOB_RUNNING = 1, FMNMF_JOB_DONE = 2, FMNMF_JOB_FAILED = 3 };
typedef struct {
  size_t hbm_budget;
  int max_active;
  int iters_per_step;
  int precision;
} fmnmf_server_opts;
fmnmf_status fmnmf_server_create(const fmnmf_server_opts* opts, fmnmf_server** out);
fmnmf_status fmnmf_server_submit(fmnmf_server* server, const void* X, int F, int T, int M, int N, int K,
                                 int n_iter, uint64_t seed, uint64_t* job);
fmnmf_status fmnmf_server_poll(fmnmf_server* server, uint64_t job, int* state, double* latency_s);
fmnmf_status fmnmf_server_wait(fmnmf_server* server, uint64_t job, double timeout_s, int* state);
fmnmf_status fmnmf_server_result(fmnmf_server* server, uint64_t job, void* out, double* loglik);
fmnmf_status fmnmf_server_stats(fmnmf_server* server, long long* queued, long long* active,
                                long long* completed, long long* failed, size_t* bytes_in_use);
fmnmf_status fmnmf_server_destroy(fmnmf_server* server);

/* Number of kernel launches this context has enqueued since creation. */
long long fmnmf_launch_count(const fmnmf_ctx* ctx);

/*
 * Log-likelihood of Eq. 17 (constant included, as fmnmf_loglik) for a state held in the
 * caller's own device buffers, computed without allocating any memory.  The paper has no
 * counterpart to this call: it is for callers that cannot call cudaMalloc - a real-time
 * audio thread that must not block (cudaMalloc may wait on the device for an unbounded
 * time), or an application whose device memory is owned entirely by its own pool
 * allocator.
 *  X, W, H, G, Q  device pointers, layouts as above (X, Q complex64; W, H, G float32).
 *  ll             device pointer to one double, written when the work completes.
 *  stream         cudaStream_t the work is enqueued on (NULL = legacy default stream);
 *                 the call is asynchronous.
 * The working memory is one static device array of 1 MiB that the library holds on every
 * device it is loaded on, until the process exits: the call rejects F > 16384 bins or
 * F*T > 117,407,744 TF bins with FMNMF_EINVAL (message via fmnmf_last_error(NULL)), and so
 * it does pointers of X, Q or ll not aligned to 8 bytes or of W, H, G not aligned to 4.
 * Every call shares that array and it keeps the last call's contents (the call clears what
 * must start at zero), so calls that overlap on the GPU race: order them on one stream or
 * with events.  The first call in a CUDA context (for the primary context: the first call
 * on a device) looks up the array's device address (cudaGetSymbolAddress, with that device
 * current) and caches it for that context; make that first call before any stream capture
 * begins on the device.  No status word is read back: a singular Q_f or a non-finite state
 * shows up as -inf or NaN in *ll.
 */
fmnmf_status fmnmf_loglik_noalloc(const void* X, const float* W, const float* H, const float* G,
                                  const void* Q, int F, int T, int M, int N, int K, double* ll,
                                  void* stream);

/* ---- FastMNMF-DP (Sec. III-B-3, Sec. III-C-3) --------------------------------------------
 * Source 0 (the paper's speech source n = 1) has the deep-prior PSD of Sec. II-B-3,
 *     lambda_ft0 = u_f v_t [sigma^2_theta(z_t)]_f,   sigma^2_theta(z) = exp(W2 tanh(W1 z + b1) + b2),
 * a two-layer decoder whose weights the caller supplies (fmnmf_dp_set_decoder; trained weights
 * are the caller's, the method does not train them).  Sources 1..N-1 (noise) have the NMF PSD
 * of Eq. 9 with K bases.  The spatial model and its updates are those of FastMNMF (Eqs. 16-21).
 * One iteration, in this order, each block from the current parameters:
 *   Z   n_proposals Metropolis proposals per frame: z' = z + sqrt(eps) xi, accepted where
 *       log u < log gamma_t, log gamma_t being the change of Eq. 17 when lambda_ft0 alone
 *       changes, with y~ of the other sources, g~ and x~ of the iteration's start;
 *   u, v the multiplicative rules of Sec. III-B-3;  W, H of the noise sources: Eqs. 23-24;
 *   g~  Eq. 21;  Q  Eqs. 18-20;  normalisation (opts.normalise): phi_f = tr(Q_f Q_f^H)/M,
 *       nu_nf = sum_m g~_nfm (into u and W), mu_0 = sum_f u_f (into v), mu_nk = sum_f w_nkf
 *       (into H); lambda g~ and the log-likelihood are unchanged by it.
 * The random draws are inputs: xi ~ N(0, I) and log u, u ~ U(0, 1), from the caller.
 * All arithmetic is FP32 on the CUDA cores; the per-bin g~ / IP kernel is that of the fused
 * FP32 schedule (float-float IP).  Layouts (row-major, float32 unless stated):
 *   X [F][T][M] complex64;  Z [T][D];  u [F];  v [T];  W [N-1][K][F];  H [N-1][K][T];
 *   G [N][F][M];  Q [F][M][M] complex64;  W1 [Hd][D];  b1 [Hd];  W2 [F][Hd];  b2 [F];
 *   xi [n_iter][n_proposals][T][D];  logu [n_iter][n_proposals][T];  images [N][F][T][M] complex64.
 * Host pointers are read or written before the call returns (copies); device pointers (with
 * the *_on_device flags) must stay valid until the work on the context's stream is done.
 * Errors: FMNMF_EINVAL for bad shapes or arguments (message via fmnmf_dp_last_error(dp), or
 * fmnmf_dp_last_error(NULL) when there is no context yet); device faults of the method
 * (singular IP system, non-finite value) are reported by the next synchronising call, as for
 * FastMNMF.  Not thread-safe per context. */
typedef struct fmnmf_dp fmnmf_dp;
typedef struct {
  int D;               /* latent dimension of z_t                      (default 16, Sec. IV-A)   */
  int Hd;              /* decoder hidden width, multiple of 4, <= 1024  (default 128)            */
  int n_proposals;     /* Metropolis proposals per frame per iteration  (default 30, Sec. IV-A)  */
  float eps;           /* proposal variance                             (default 1e-4, Sec. IV-A)*/
  int normalise;       /* 1: scale normalisation                        (default 1)              */
  void* stream;        /* cudaStream_t for all device work; NULL = a private stream               */
} fmnmf_dp_opts;

fmnmf_status fmnmf_dp_default_opts(fmnmf_dp_opts* opts);
/* Needs 1 <= N <= 8, (N-1) K <= 256, N M small enough for the per-bin kernel of the fused
 * schedule, and one frame's x~, y~ and decoder staging within the device's shared memory. */
fmnmf_status fmnmf_dp_create(fmnmf_dp** out, const void* X, int x_on_device, int F, int T, int M, int N,
                             int K, const fmnmf_dp_opts* opts);
/* Host weights; finite.  Invalidates the state (r = sigma^2(z) changes): set it again. */
fmnmf_status fmnmf_dp_set_decoder(fmnmf_dp* dp, const float* W1, const float* b1, const float* W2,
                                  const float* b2);
/* Host state; u, v, W, H finite and positive, G finite and nonnegative, Q finite.  Forms r and
 * lambda of every source, x~, log|det Q|^2 and the log-likelihood; resets the accepted count.
 * W and H may be NULL when N = 1. */
fmnmf_status fmnmf_dp_set_state(fmnmf_dp* dp, const float* Z, const float* u, const float* v,
                                const float* W, const float* H, const float* G, const void* Q);
/* Host copies of the state; any pointer may be NULL.  Synchronises. */
fmnmf_status fmnmf_dp_get_state(fmnmf_dp* dp, float* Z, float* u, float* v, float* W, float* H,
                                float* G, void* Q);
/* n_iter iterations, enqueued (asynchronous); the log-likelihood of the state after the last
 * one is ready at the next fmnmf_dp_loglik.  Host draws are copied in chunks. */
fmnmf_status fmnmf_dp_iterate(fmnmf_dp* dp, int n_iter, const float* xi, const float* logu,
                              int draws_on_device);
/* The Z block alone (one iteration's n_proposals proposals per frame) with the current u, v,
 * W, H, g~, Q and x~; writes log gamma of every proposal to loggamma [n_proposals][T] (host,
 * may be NULL) and the number accepted to *accepted (may be NULL).  The log-likelihood is not
 * refreshed.  Synchronises. */
fmnmf_status fmnmf_dp_metropolis(fmnmf_dp* dp, const float* xi, const float* logu, int draws_on_device,
                                 float* loggamma, long long* accepted);
fmnmf_status fmnmf_dp_sync(fmnmf_dp* dp);
fmnmf_status fmnmf_dp_loglik(fmnmf_dp* dp, double* ll);
/* Proposals accepted since the last fmnmf_dp_set_state. */
fmnmf_status fmnmf_dp_accepted(fmnmf_dp* dp, long long* n);
/* Multichannel Wiener filter (Eq. 3 with Eq. 16) of every source, as fmnmf_separate. */
fmnmf_status fmnmf_dp_separate(fmnmf_dp* dp, void* out, int out_on_device);
fmnmf_status fmnmf_dp_destroy(fmnmf_dp* dp);
const char* fmnmf_dp_last_error(const fmnmf_dp* dp);

#ifdef __cplusplus
}
#endif

#endif /* FASTMNMF_H */
