/*
 * srmra.h -- C ABI of libsrmra.so: projected expectation-maximization for 2D
 * super-resolution multi-reference alignment (SR-MRA) on one NVIDIA GB300 (sm_103a).
 *
 * Method: Shani, Tirer, Giryes, Bendory, "Denoiser-based projections for 2D
 * super-resolution MRA" (arXiv 2204.04754).  Section references below are to that
 * paper.
 *
 * Data model (Sec. 1, Eq. 1):  y_i = P R_{s_i} x + eps_i,  i = 0..N-1, where
 *   x      is the L x L high-resolution image (L = L_high),
 *   R_s    is the 2D circular translation (R_s x)[q1,q2] = x[q1-s1, q2-s2] (mod L),
 *   P      keeps the l x l samples z[n1*K, n2*K], l = L / K (K integer),
 *   eps_i  is i.i.d. N(0, sigma^2) noise, s1 ~ rho1, s2 ~ rho2 i.i.d.
 * The shift index is s = s1 * L + s2 with s1 acting on the first (row) axis.
 *
 * One EM iteration (Sec. 2, Eqs. weights_EM, x_EM, rho_EM) maps theta_t = (x, rho1,
 * rho2) to theta_{t+1}:
 *   w[i,s]  = rho1[s1] rho2[s2] exp(-||y_i - P R_s x||^2 / (2 sigma^2)) / C_i,
 *   x_{t+1} = b / A with b = sum_{i,s} w R_s^T P^T y_i and A the diagonal of
 *             sum_{i,s} w R_s^T P^T P R_s (P^{-1} in the paper read as P^T); a pixel
 *             with A = 0 keeps its value,
 *   rho[s]  = sum_i w[i,s] / sum_{i,s'} w[i,s'], rho1 / rho2 its marginals,
 *   LL(theta_t) = sum_i log sum_s rho[s] exp(-||y_i - P R_s x||^2 / (2 sigma^2))
 *             (Eq. likelihood_EM without its Gaussian constant).
 * Projected EM (Algorithm 2) applies a denoiser x <- D(x, sigma_BM) after every F
 * EM steps and decays sigma_BM_t = 2^{-1/10} sigma_BM_{t-1} (Eq. decaying_function).
 *
 * Conventions for every entry point:
 *   - Arrays are C-contiguous.  y is N x l x l float32 (y[i][n1][n2]); x is L x L
 *     float32 (x[q1][q2]); rho1 (indexed by s1) and rho2 (by s2) are float64, length L.
 *   - "host" pointers are ordinary CPU memory (pinned or pageable); "device" pointers
 *     are CUDA global memory on the context's device.
 *   - Every call returns srmra_status; no C++ exception crosses this ABI.  On an error
 *     the context state is unchanged unless the entry point says otherwise, and
 *     srmra_last_error() returns a message.
 *   - There is no CPU fallback: without a usable sm_103a GPU every call that needs one
 *     returns SRMRA_ECUDA.
 *   - Work is enqueued on the CUDA stream given at creation.  Entry points that return
 *     host values (log-likelihoods, state) synchronise that stream; the others do not.
 */
#ifndef SRMRA_H
#define SRMRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct srmra_ctx srmra_ctx; /* opaque; owned by the library */

typedef enum {
  SRMRA_OK = 0,
  SRMRA_EINVAL = 1,   /* invalid argument (shape, sigma, rho not on the simplex, ...) */
  SRMRA_ENOMEM = 2,   /* device or host allocation failed */
  SRMRA_ECUDA = 3,    /* CUDA error, or no usable sm_103a device */
  SRMRA_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  SRMRA_ENUMERIC = 5, /* NaN / Inf met in the log-likelihood, x or rho */
  SRMRA_EBUSY = 6     /* context in use by a batched call */
} srmra_status;

/* Arithmetic of the two contractions <y_i, P R_s x> and sum_i w y_i.
 *   SRMRA_FP32   : float32 CUDA-core FMA (the plain form).
 *   SRMRA_BF16   : bf16 tensor-core operands, float32 accumulation and softmax.
 *   SRMRA_BF16X3 : split-bf16 (hi + lo) for the cross term, hi*hi + hi*lo + lo*hi on
 *                  tensor cores with float32 accumulation; fp16 weights (scaled by
 *                  2^12) and fp16 y' for the M-step sum.
 *   SRMRA_FFT32  : float32 polyphase-FFT form.  Per sub-image x_r of the K^2
 *                  polyphase components, <y_i, P R_s x> over all lags t of phase r
 *                  is the circular cross-correlation of y_i with x_r (Sec. 2, the
 *                  structure behind Theorem 1), computed with l x l FFTs; the M-step
 *                  right-hand side of Eq. (x_EM) likewise.  Same results as the
 *                  dense forms up to rounding, O(N K^2 l^2 log l) instead of
 *                  O(N L^2 l^2) flops.  Needs l = L/K in {8, 16, 32}; srmra_create
 *                  returns SRMRA_EINVAL otherwise.
 * The global log-likelihood is reduced in float64 in every form. */
typedef enum {
  SRMRA_FP32 = 0,
  SRMRA_BF16 = 1,
  SRMRA_BF16X3 = 2,
  SRMRA_FFT32 = 3
} srmra_precision;

/* flags */
#define SRMRA_FLAG_CHECK_NUMERIC 1u /* scan x, rho, LL for NaN/Inf after each iteration */
#define SRMRA_FLAG_NO_CLUSTER 2u    /* tensor-core forms: recompute the weights per pixel
                                       chunk instead of sharing them across a cluster */
/* SRMRA_BF16X3: the M-step sum Z' = W^T Y' runs on fp16 operands.  With one fp16 part
 * per operand its rounding (2^-11 relative) averages out only over many observations;
 * below about N = 31.25 (L/K) max(1, 2 sigma) observations the library therefore splits
 * both operands into fp16 hi + lo parts (three MMAs, per-chunk kernel): the compensated
 * M-step.  These flags force it on, or off. */
#define SRMRA_FLAG_MSTEP_COMP 4u
#define SRMRA_FLAG_MSTEP_FP16 8u
/* Tensor-core forms: pass 1 uses 128-shift tiles (four TMEM accumulators) instead of
 * 256-shift tiles (two); a batch's autotuner also chooses between them. */
#define SRMRA_FLAG_P1_TILE128 16u
/* SRMRA_BF16X3 with up to four 256-pixel chunks (L/K <= 32): pass 2 in the pair form,
 * 2-CTA tensor-core MMAs (cta_group::2) on two shift tiles at once, one per CTA of a
 * pair (clusters of 2G CTAs for G chunks). */
#define SRMRA_FLAG_P2_PAIR 32u

typedef struct {
  int32_t L_high;  /* L >= 2 */
  int32_t K;       /* down-sampling factor, K >= 1, K divides L */
  int64_t N;       /* number of observations, N >= 1 */
  double sigma;    /* noise standard deviation, sigma > 0 */
  int32_t prec;    /* srmra_precision */
  uint32_t flags;  /* SRMRA_FLAG_* */
} srmra_params;

/* A user denoiser D(x, sigma_BM) for srmra_project / srmra_solve.  x_dev is the L x L
 * float32 image in device memory, valid only during the call; the callback must
 * enqueue its work on `stream` (a cudaStream_t) and return 0 on success.  A non-zero
 * return makes the calling entry point fail with SRMRA_EINVAL. */
typedef int32_t (*srmra_denoiser_fn)(float* x_dev, int32_t L, double sigma_bm,
                                     void* stream, void* user);

/* srmra_create -- allocate a context for one SR-MRA problem (Eq. 1).
 *   p          : problem sizes and options.  EINVAL if K does not divide L, sigma <= 0,
 *                N < 1, L < 2 or prec is unknown.
 *   y          : N x l x l float32 observations; host memory if y_is_device == 0,
 *                device memory otherwise.  The library copies them into its own
 *                device buffers (and derives the layouts its kernels read); the
 *                caller keeps ownership of y and may free it after the call.
 *   x0         : L x L float32 initial image (host), or NULL for the nearest-neighbour
 *                upsampling of the mean observation.
 *   rho1_0/2_0 : length-L float64 initial distributions (host), or NULL for uniform.
 *                EINVAL if an entry is negative or the sum is off 1 by more than 1e-6;
 *                otherwise they are renormalised.
 *   cuda_stream: cudaStream_t on which all work is enqueued (NULL = legacy default).
 *   out        : receives the context.  Device memory is held until srmra_destroy.
 * Errors: EINVAL, ENOMEM (device allocation), ECUDA.  *out is NULL on error. */
srmra_status srmra_create(const srmra_params* p, const float* y, int32_t y_is_device,
                          const float* x0, const double* rho1_0, const double* rho2_0,
                          void* cuda_stream, srmra_ctx** out);

/* srmra_em_iter -- run n_iters EM iterations theta_t -> theta_{t+1} (Sec. 2, Eqs.
 * weights_EM, x_EM, rho_EM), without projection.
 *   loglik_out : host array of n_iters float64 receiving LL(theta_t) of each iteration
 *                (the likelihood of the parameters the E-step used), or NULL.  When it
 *                is non-NULL the call synchronises the stream and also checks the
 *                device status word (ETIMEOUT / ENUMERIC).
 * Errors: EINVAL (n_iters < 0), ECUDA, ETIMEOUT, ENUMERIC. */
srmra_status srmra_em_iter(srmra_ctx* ctx, int32_t n_iters, double* loglik_out);

/* srmra_project -- x <- D(x, sigma_bm) (Algorithm 2, step 2).  fn == NULL selects the
 * built-in denoiser: non-overlapping 8 x 8 blocks anchored at pixel (0,0), orthonormal
 * 2D DCT-II in float64, DC coefficient kept, an AC coefficient kept iff
 * |c| > 2.7 * sigma_bm, inverse DCT.  The built-in denoiser needs L % 8 == 0 (EINVAL
 * otherwise).  Does not change the context's sigma_BM. */
srmra_status srmra_project(srmra_ctx* ctx, double sigma_bm, srmra_denoiser_fn fn,
                           void* user);

/* Built-in denoiser variants (srmra_set_denoiser). */
#define SRMRA_DENOISE_HARD 0 /* keep an AC coefficient iff |c| > threshold * sigma_BM */
#define SRMRA_DENOISE_SOFT 1 /* c <- sign(c) max(|c| - t, 0): the prox of t ||AC||_1, a
                                convex prox as in Sec. 4's Assumption 2 */

/* srmra_set_denoiser -- choose the built-in denoiser used by srmra_project,
 * srmra_solve and batches: mode SRMRA_DENOISE_HARD (default) or _SOFT, threshold
 * multiplier of sigma_BM (default 2.7), and spin != 0 to average the block denoiser
 * over all 64 offsets of the 8 x 8 block grid (cycle spinning; allocates 64 L^2
 * float64 of device memory once).  The paper's BM3D (Sec. 5) is not part of the
 * method; any other denoiser can be passed as a callback. */
srmra_status srmra_set_denoiser(srmra_ctx* ctx, int32_t mode, double threshold, int32_t spin);

/* srmra_solve -- Algorithm 2 (projected EM) for `iters` EM iterations: after every
 * iteration whose 1-based global count t+1 is a multiple of F, apply D(x, sigma_BM)
 * (fn, or the built-in DCT denoiser if fn == NULL) and set sigma_BM <- decay * sigma_BM
 * (Eq. decaying_function uses decay = 2^{-1/10}).  F == 0 runs plain EM.
 * sigma_bm1 > 0 resets the context's sigma_BM to sigma_bm1 first (Eq. decaying_function
 * starts at sigma_BM_1 = 1); sigma_bm1 <= 0 continues from the stored sigma_BM (resume).
 * loglik_out: host array of `iters` float64 (LL(theta_t) per iteration) or NULL. */
srmra_status srmra_solve(srmra_ctx* ctx, int32_t iters, int32_t F, double sigma_bm1,
                         double decay, srmra_denoiser_fn fn, void* user,
                         double* loglik_out);

/* srmra_get_state -- copy the current estimate to host buffers (any may be NULL):
 * x (L*L float32), rho1, rho2 (L float64 each), sigma_BM, iteration count t.
 * Synchronises the stream. */
srmra_status srmra_get_state(srmra_ctx* ctx, float* x, double* rho1, double* rho2,
                             double* sigma_bm, int32_t* t);

/* srmra_set_state -- replace the estimate (checkpoint resume).  x: L*L float32 host;
 * rho1, rho2: L float64 host (validated as in srmra_create); sigma_bm and t are stored
 * as given.  Resuming from a state returned by srmra_get_state reproduces the
 * uninterrupted run bit for bit (all reductions have a fixed order). */
srmra_status srmra_set_state(srmra_ctx* ctx, const float* x, const double* rho1,
                             const double* rho2, double sigma_bm, int32_t t);

/* srmra_get_lse -- diagnostics of the last E-step: lse[i] = log sum_s rho[s]
 * exp(-||y_i - P R_s x||^2 / (2 sigma^2)) (float64, N entries, host) and/or the
 * per-shift weight sums c[s] = sum_i w[i,s] (float64, L*L entries, host).  Either
 * pointer may be NULL.  EINVAL before the first iteration.  Synchronises. */
srmra_status srmra_get_estep(srmra_ctx* ctx, double* lse, double* c);

/* ---- Data-parallel decomposition over the observations (one all-reduce per iteration).
 * The M-step of Eqs. (x_EM), (rho_EM) reads only sums over observations: per shift s
 * c_s = sum_i w[i,s] and zb_s = sum_i w[i,s] ybar_i, per sub-image r and low-resolution
 * pixel m the back-projection b'_r[m] of the centred observations, and LL = sum_i lse_i.
 * Shards of the observations (contexts holding disjoint subsets, all at the same theta)
 * therefore produce statistics that add, and the M-step of their sum is the EM iteration
 * of the union.  The vector layout (float64, srmra_stats_length() entries):
 *   [c_s (L^2, s = s1 L + s2) | zb_s (L^2) | b'_r[m] (K^2 l^2 = L^2, index r l^2 + m,
 *    r = r1 K + r2) | LL (1)].
 * Sums are in the centred form of the context: y'_i = y_i - ybar_i, so shards must come
 * from the same problem (same L, K, sigma); ybar_i is per observation, so any split of
 * the observations is valid. */

/* srmra_stats_length -- entries of the statistics vector, 3 L^2 + 1. */
srmra_status srmra_stats_length(const srmra_ctx* ctx, int64_t* len);

/* srmra_estep_stats -- the E-step (both passes) at the context's theta over its
 * observations, reduced to the statistics vector.  stats: host memory (the call
 * synchronises and checks the device status word) or, with stats_is_device != 0, device
 * memory on the context's device, written in stream order without synchronising. */
srmra_status srmra_estep_stats(srmra_ctx* ctx, double* stats, int32_t stats_is_device);

/* srmra_mstep_stats -- the M-step (Eqs. x_EM, rho_EM) from a statistics vector (for
 * example the sum over shards): theta_t -> theta_{t+1} in this context, t += 1.  Then
 * Algorithm 2 on the context's own schedule (srmra_set_schedule; none by default): if
 * its F > 0 and t is a multiple of F, the built-in denoiser x <- D(x, sigma_BM) and
 * sigma_BM <- decay sigma_BM (Eq. decaying_function), so that every rank of a sharded
 * solve projects identically.  stats: host, or device memory read in the context's
 * stream order (the caller orders any producer, e.g. a collective on another stream,
 * before this call).  loglik_out (host, may be NULL): the LL entry of the vector;
 * given, the call synchronises and checks the status word (ENUMERIC). */
srmra_status srmra_mstep_stats(srmra_ctx* ctx, const double* stats, int32_t stats_is_device,
                               double* loglik_out);

/* srmra_launch_count -- number of CUDA kernels this context has launched so far. */
srmra_status srmra_launch_count(const srmra_ctx* ctx, int64_t* count);

/* srmra_set_wait_limit -- limit, in nanoseconds, of the bounded device-side waits of
 * this context's tensor-core kernels (mbarrier, mailbox and flag waits; default 2e9).
 * A wait that runs out makes its kernel stop the pipeline, drain its own asynchronous
 * copies and MMAs, release TMEM and set the device status word: the next entry point
 * that reads the status (one returning host values, or any call with
 * SRMRA_FLAG_CHECK_NUMERIC) returns SRMRA_ETIMEOUT, and the GPU keeps answering.
 * limit_ns must lie in [1e3, 6e10].
 * test_hook exists to test that failure path (0 in normal use): 1 makes the epilogue
 * of the first CTA of pass 1 wait on a barrier that nothing completes; 2 does the same
 * in pass 2 (in a cluster form the first cluster's rank 0, so that its peers' waits for
 * its weight tile run out as well).  The wait runs out after limit_ns and the iteration
 * reports SRMRA_ETIMEOUT; x and rho are then undefined until srmra_set_state.
 * A batch copies the setting when it is created; a grouped launch uses its first
 * problem's.  The float32 and FFT forms have no such waits (the setting is kept,
 * unused).  Errors: SRMRA_EINVAL. */
srmra_status srmra_set_wait_limit(srmra_ctx* ctx, int64_t limit_ns, int32_t test_hook);

/* Pass-2 kernel forms reported by srmra_get_plan (entry 4). */
#define SRMRA_P2_PER_CHUNK 0   /* tensor cores, weights recomputed per 256-pixel chunk */
#define SRMRA_P2_RING 1        /* tensor cores, ring cluster form (clusters of 2-4) */
#define SRMRA_P2_INTERLEAVED 2 /* tensor cores, interleaved cluster form (clusters of 5-16) */
#define SRMRA_P2_FP32 3        /* float32 persistent clusters */
#define SRMRA_P2_FFT 4         /* polyphase-FFT form */
#define SRMRA_P2_PER_CHUNK_COMP 5 /* tensor cores, per chunk, compensated M-step (bf16x3) */
#define SRMRA_P2_PAIR 6        /* tensor cores, 2-CTA MMAs, clusters of 2-8 (bf16x3) */

/* srmra_get_plan -- the work decomposition the context's kernels use (no computation;
 * the executed-work counts of a profile are derived from it).  out (host, n int32
 * entries, n <= 7 are filled): [0] pass-1 shift groups per observation tile, [1] pass-1
 * shift tiles per group, [2] pass-2 cluster size G (CTAs sharing each weight tile; 1 =
 * none; the pair form: pairs per cluster), [3] pass-2 chunk groups (each recomputes
 * the logits of a shift tile), [4] the pass-2 form (SRMRA_P2_*), [5] pass-2 observation
 * splits, [6] shifts per pass-1 tile of the tensor-core forms (256 or 128; 0 for the
 * others).  Errors: SRMRA_EINVAL. */
srmra_status srmra_get_plan(const srmra_ctx* ctx, int32_t* out, int32_t n);

/* ---- Batches: many independent problems advanced together (one GPU). ----
 * A batch groups contexts of the same precision form and CUDA stream.  Each EM
 * iteration (Sec. 2) of a batch runs ONE grouped persistent launch of pass 1 and ONE of
 * pass 2 over the work units of all its problems (tensor-core forms; the float32 form
 * launches per problem), plus the small per-problem kernels; the whole iteration,
 * including the projection step of Algorithm 2, is captured once into a CUDA graph and
 * replayed.  Problems keep their own data, estimate and schedule; results do not depend
 * on which other problems share the batch beyond float32 rounding of the chosen work
 * decomposition. */
typedef struct srmra_batch srmra_batch; /* opaque; owned by the library */

#define SRMRA_BATCH_AUTOTUNE 1u /* time candidate work decompositions, keep the fastest */
#define SRMRA_BATCH_NO_GRAPH 2u /* enqueue kernels directly instead of a CUDA graph */

/* srmra_batch_create -- build a batch over ctxs[0..count-1] (distinct, same precision,
 * same stream).  The contexts stay owned by the caller and must outlive the batch; a
 * context may belong to several batches but batches that share a context must not run
 * concurrently.  With SRMRA_BATCH_AUTOTUNE the tile shape and work decomposition of the
 * grouped launches (pass-1 tiles of 256 or 128 shifts x shift groups of pass 1 x {1,2}
 * x observation ranges of pass 2 x {1,2} x problem order {as given, most expensive unit
 * first}) are timed on the device and the fastest is kept (the problems' estimates are
 * not changed by the timing runs; the contexts keep the chosen plan).  Without it the
 * contexts must share one pass-1 tile width (SRMRA_FLAG_P1_TILE128).
 * Errors: EINVAL, ENOMEM, ECUDA.  Message: srmra_batch_last_error(NULL). */
srmra_status srmra_batch_create(srmra_ctx** ctxs, int32_t count, uint32_t flags,
                                srmra_batch** out);

/* srmra_batch_solve -- `iters` iterations of Algorithm 2 for every problem of the batch:
 * each problem projects with the built-in denoiser after every iteration whose 1-based
 * count (its own t+1) is a multiple of F (F = 0: plain EM) and then decays its sigma_BM
 * by `decay`.  sigma_bm1 > 0 resets every problem's sigma_BM first.  loglik_last: host
 * array of `count` float64 (order of srmra_batch_create) receiving LL(theta) of each
 * problem's last iteration, or NULL.  Synchronises the stream. */
srmra_status srmra_batch_solve(srmra_batch* b, int32_t iters, int32_t F, double sigma_bm1,
                               double decay, double* loglik_last);

/* (srmra_batch_solve with F < 0 uses every problem's own schedule, see
 * srmra_set_schedule, instead of one F and decay for all.) */

/* srmra_set_schedule -- the Algorithm 2 schedule of this problem: projection every F
 * iterations (F = 0: none), current sigma_BM, and the decay factor applied after each
 * projection (Eq. decaying_function).  Used by srmra_mstep_stats and by a batch solved
 * with F < 0.  EINVAL if F < 0, sigma_bm < 0, decay <= 0, or F > 0 with L % 8 != 0. */
srmra_status srmra_set_schedule(srmra_ctx* ctx, int32_t F, double sigma_bm, double decay);

/* srmra_estimate_device_bytes -- device memory srmra_create would allocate for these
 * parameters (no device memory is touched; for admission control). */
srmra_status srmra_estimate_device_bytes(const srmra_params* p, int64_t* bytes);

/* srmra_device_bytes -- device memory held by a context. */
srmra_status srmra_device_bytes(const srmra_ctx* ctx, int64_t* bytes);

/* srmra_batch_tuning -- the decomposition chosen by the autotuner (scales 1 or 2, order
 * 0 = as given, 1 = most expensive first) and its timed milliseconds per pass pair. */
srmra_status srmra_batch_tuning(const srmra_batch* b, int32_t* p1_scale, int32_t* p2_scale,
                                int32_t* order, double* ms);

/* srmra_batch_tiles -- the tile shape the batch's grouped pass-1 launch uses: its shift
 * width (256 or 128; chosen by the autotuner with SRMRA_BATCH_AUTOTUNE, else the
 * contexts' own).  Errors: SRMRA_EINVAL. */
srmra_status srmra_batch_tiles(const srmra_batch* b, int32_t* p1_shift_tile);

/* srmra_batch_pass_ms -- device time (CUDA events) of the grouped pass-1 and pass-2
 * launches of the batch's most recent iteration.  Synchronises the stream. */
srmra_status srmra_batch_pass_ms(srmra_batch* b, double* ms_pass1, double* ms_pass2);

void srmra_batch_destroy(srmra_batch* b);
const char* srmra_batch_last_error(const srmra_batch* b);

/* srmra_em_iter_batch -- n_iters plain EM iterations (no projection) of every context,
 * through a transient batch (no autotuning, no graph). */
srmra_status srmra_em_iter_batch(srmra_ctx** ctxs, int32_t count, int32_t n_iters);

/* ---- Serving: continuous batching of solve requests on one GPU. ----
 * srmra_server_submit queues a request (a full projected-EM solve of one problem: y on
 * the host, copied at submission; optional x0; iteration count; Algorithm 2 schedule F,
 * sigma_BM_1, decay).  Each srmra_server_step admits queued requests in arrival order
 * while a slot is free and their device memory (srmra_estimate_device_bytes) fits the
 * budget -- their observations, x and rho then stay on the device until they retire --,
 * advances every running request by one EM iteration (+ scheduled projection) as one
 * batch (grouped launches, CUDA graph re-captured only when the set of requests
 * changes), and retires the requests that reached their iteration count (estimate
 * copied to the host, device memory released).  Requests submitted while others run
 * join at the next iteration boundary.  A request's arithmetic is independent of the
 * other requests, so its result equals srmra_create + srmra_solve of the same problem.
 * Submission may come from another thread than the one calling srmra_server_step. */
typedef struct srmra_server srmra_server;

/* prec: the form every request runs in (srmra_precision), or SRMRA_SERVER_AUTO: each
 * request runs in the polyphase-FFT form when L/K is 8, 16 or 32 (faster and more
 * accurate than the tensor-core forms there) and in SRMRA_BF16X3 otherwise; the server
 * then keeps one batch per form and advances them in turn each step. */
#define SRMRA_SERVER_AUTO 4
srmra_status srmra_server_create(int64_t device_budget_bytes, int32_t max_active,
                                 int32_t prec, void* cuda_stream, srmra_server** out);

/* y: N x l x l float32 host array (p->N, p->L_high, p->K, p->sigma; p->prec is replaced by
 * the server's form, or by the form SRMRA_SERVER_AUTO picks); x0: L x L float32 host or NULL (mean-upsampled init).  ENOMEM if
 * the request alone exceeds the budget.  *request_id identifies it. */
srmra_status srmra_server_submit(srmra_server* s, const srmra_params* p, const float* y,
                                 const float* x0, int32_t iters, int32_t F, double sigma_bm1,
                                 double decay, int64_t* request_id);

/* One admission + iteration + retirement round; reports the numbers of running and
 * queued requests afterwards and of requests that finished in this step. */
srmra_status srmra_server_step(srmra_server* s, int32_t* n_running, int32_t* n_queued,
                               int32_t* n_finished);

/* state: 0 queued, 1 running, 2 done, 3 failed (the call then returns the failure).
 * When done, x (L*L float32), rho1, rho2 (L float64) and the last iteration's
 * log-likelihood are copied out (any pointer may be NULL).  times_ms (3 doubles or
 * NULL): submit->admit, admit->done, submit->done in milliseconds (-1 if not yet). */
srmra_status srmra_server_result(srmra_server* s, int64_t id, int32_t* state, float* x,
                                 double* rho1, double* rho2, double* loglik_last,
                                 double* times_ms);

/* Device memory reserved by running requests, and the budget. */
srmra_status srmra_server_memory(srmra_server* s, int64_t* used, int64_t* budget);

void srmra_server_destroy(srmra_server* s);
const char* srmra_server_last_error(const srmra_server* s);

/* Phases of one iteration, for srmra_profile_read. */
enum {
  SRMRA_PHASE_PREP = 0,     /* sub-image statistics, logit column terms, templates */
  SRMRA_PHASE_PASS1 = 1,    /* logits + online log-sum-exp partials */
  SRMRA_PHASE_COMBINE = 2,  /* per-observation lse, float64 log-likelihood partials */
  SRMRA_PHASE_PASS2 = 3,    /* recomputed weights -> M-step partial sums */
  SRMRA_PHASE_FINAL = 4,    /* rho, coverage, x = b / A */
  SRMRA_PHASE_DENOISE = 5,  /* built-in denoiser */
  SRMRA_NUM_PHASES = 6
};

/* srmra_profile -- enable (1) or disable (0) per-phase timing: CUDA events are recorded
 * on the context's stream around every phase launched from now on. */
srmra_status srmra_profile(srmra_ctx* ctx, int32_t enable);

/* srmra_profile_read -- synchronise, then add the device time (ms) and launch count of
 * every recorded phase since the last read into ms[p] and count[p] (arrays of
 * SRMRA_NUM_PHASES, host, either may be NULL), and clear the records. */
srmra_status srmra_profile_read(srmra_ctx* ctx, double* ms, int64_t* count);

/* ---- Online (mini-batch) EM over shards of the observations. ----
 *
 * The paper points to online strategies to cut the cost of the likelihood term for
 * large N (Sec. 6) without fixing an algorithm; this is mini-batch EM with
 * stochastic-approximation sufficient statistics.  The observations are split into
 * shard contexts (created with srmra_create, device resident; same L, K, sigma,
 * precision and stream).  The online object holds the estimate theta = (x, rho1,
 * rho2) and the running statistics S of Eqs. (x_EM), (rho_EM): per shift
 * c_s = sum_i w^{i,s} and zb_s = sum_i w^{i,s} ybar_i, per low-resolution pixel of
 * every sub-image the back-projection b' of the centred observations.  A step on
 * shard k:
 *   1. E-step of the current theta over shard k's n_k observations (both passes),
 *   2. S <- (1 - gamma) S + gamma (shard statistics) / n_k   (the first step uses 1),
 *   3. the M-step of Eqs. (x_EM), (rho_EM) on S.
 * A single shard holding all observations with gamma = 1 is one EM iteration.
 * The shards' own x / rho are overwritten by each step that uses them.            */
typedef struct srmra_online srmra_online;

/* srmra_online_create -- shards: n_shards distinct contexts (kept by the caller, not
 * owned; they must outlive the online object).  x0, rho1_0, rho2_0: host, or NULL for
 * shard 0's current state.  Errors: SRMRA_EINVAL (mismatched shards, bad rho). */
srmra_status srmra_online_create(srmra_ctx* const* shards, int32_t n_shards, const float* x0,
                                 const double* rho1_0, const double* rho2_0,
                                 srmra_online** out);

/* srmra_online_step -- one step on shard `shard` with step size gamma in (0, 1].
 * loglik_out (host, may be NULL): the shard's log-likelihood sum_i lse_i at the theta
 * the step started from (Eq. likelihood_EM over the batch).  Synchronous when
 * loglik_out is given; otherwise only enqueued. */
srmra_status srmra_online_step(srmra_online* on, int32_t shard, double gamma, double* loglik_out);

/* srmra_online_project -- x <- D(x, sigma_bm) with the built-in block-DCT denoiser
 * (the settings of srmra_set_denoiser on shard 0; needs L % 8 == 0). */
srmra_status srmra_online_project(srmra_online* on, double sigma_bm);

/* srmra_online_get_state -- current estimate to host buffers (any may be NULL). */
srmra_status srmra_online_get_state(srmra_online* on, float* x, double* rho1, double* rho2,
                                    int64_t* steps_done);

void srmra_online_destroy(srmra_online* on);
const char* srmra_online_last_error(const srmra_online* on);

/* ---- Projected method of moments (Algorithm 1). ----
 *
 * Estimates theta = (x, rho1, rho2) from the first two moments of the observations,
 * which a MoM object computes once from a context's device-resident observations
 * (Eq. empiric_MOM with D = 2): M1^ = (1/N) sum_i y_i and M2^ = (1/N) sum_i y_i y_i^T,
 * both over the flattened l x l images (float32 products, float64 partial sums).
 * The model's moments at theta, with t_s = P R_s x and rho_s = rho1[s1] rho2[s2]
 * (Sec. 2), are M1 = sum_s rho_s t_s and M2 = sum_s rho_s t_s t_s^T + sigma^2 I, and
 * the objective is Eq. (LS_SR):
 *   f = ||M2 - M2^||_F^2 + lambda ||M1 - M1^||^2,   lambda = 1 / (L^2 (1 + sigma^2)).
 * Its gradient, with R = M2 - M2^ and r = M1 - M1^:
 *   df/drho_s = 2 t_s^T R t_s + 2 lambda t_s^T r,
 *   df/drho1  = G rho2, df/drho2 = G^T rho1   (G[s1][s2] = df/drho_s),
 *   df/dx     = sum_s rho_s (P R_s)^T (4 R t_s + 2 lambda r).
 * A step of srmra_mom_run is the fixed-step projected gradient iteration the paper
 * analyses (Sec. 4, Eq. pgm) in place of the F BFGS steps of Algorithm 1:
 *   x <- x - mu_x df/dx,  rho1, rho2 <- Euclidean projections onto the probability
 *   simplex of rho - mu_rho df/drho (both gradients taken at the same theta),
 * and after every F-th step x <- D(x, sigma_BM), sigma_BM <- decay sigma_BM
 * (Eq. decaying_function).  The estimate lives in the context: srmra_mom_run starts
 * from the context's x, rho1, rho2 and leaves its result there (srmra_get_state). */
typedef struct srmra_mom srmra_mom;

/* srmra_mom_create -- bind to ctx (not owned; it must outlive the MoM object), allocate
 * the moment buffers (about 4 (3 + splits) l^4 + 12 L^2 l^2 bytes, l^2 rounded up to
 * 128) and compute the empirical moments (synchronous).  Needs L <= 1024 and
 * (L/K)^2 <= 8192.  Errors: SRMRA_EINVAL, SRMRA_ENOMEM, SRMRA_ECUDA. */
srmra_status srmra_mom_create(srmra_ctx* ctx, srmra_mom** out);

/* srmra_mom_moments -- copy M1^ (l^2 float64) and M2^ (l^2 x l^2 float64, row-major) to
 * host buffers; either may be NULL.  Synchronous. */
srmra_status srmra_mom_moments(srmra_mom* m, double* M1h, double* M2h);

/* srmra_mom_eval -- f and its gradient at the context's current theta into host
 * buffers (any may be NULL): f (1), gx (L x L, row-major), g1 = df/drho1 (L),
 * g2 = df/drho2 (L).  Synchronous.  SRMRA_ENUMERIC if f is not finite. */
srmra_status srmra_mom_eval(srmra_mom* m, double* f, double* gx, double* g1, double* g2);

/* srmra_mom_run -- iters steps (above).  F = 0: no denoiser; fn == NULL selects the
 * built-in denoiser of srmra_project (needs L % 8 == 0), else fn(user) is called as
 * there.  f_out (host, iters float64, may be NULL): f at the theta each step started
 * from.  Synchronous.  Errors: SRMRA_EINVAL (arguments, denoiser), SRMRA_ENUMERIC. */
srmra_status srmra_mom_run(srmra_mom* m, int32_t iters, int32_t F, double mu_x, double mu_rho,
                           double sigma_bm1, double decay, srmra_denoiser_fn fn, void* user,
                           double* f_out);

/* srmra_mom_recompute_moments -- enqueue the empirical-moment pass again (the
 * observations are unchanged, so the result is the same; for timing the one-pass
 * data-parallel part). */
srmra_status srmra_mom_recompute_moments(srmra_mom* m);

void srmra_mom_destroy(srmra_mom* m);
const char* srmra_mom_last_error(const srmra_mom* m);

/* srmra_loglik_noalloc -- per-observation log-likelihood terms without any device
 * allocation.  The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc -- services that size all device memory once at start-up so
 * that no request can fail later on an allocation, host code that must not block on
 * the allocator (cudaMalloc can synchronise the device), and embedders whose own
 * allocator owns every byte of device memory.
 *
 * It computes the same values as the E-step of srmra_em_iter in the float32 form:
 *   lse[i] = log sum_s rho1[s1] rho2[s2] exp(-||y_i - P R_s x||^2 / (2 sigma^2)),
 *   *ll    = sum_i lse[i]   (float64, fixed reduction order).
 * Inputs (device memory, caller-owned): y (N x l x l float32), x (L x L float32),
 * rho1, rho2 (L float64, on the simplex).  Outputs (device memory, caller-owned): lse
 * (N float64) and ll (1 float64).  Work is enqueued on cuda_stream; the call does not
 * synchronise.
 *
 * Intermediate buffers live in one fixed device array of srmra_noalloc_scratch_bytes()
 * bytes (64 MiB) per device, which every device that loads the library holds until the
 * process exits.  Problems whose intermediates do not fit return SRMRA_EINVAL with a
 * message (srmra_noalloc_last_error); roughly N * l^2 <= 7.5e6 fits.  The library calls
 * no cudaMalloc, cudaFree or allocating routine here.  The first call on a device looks
 * up the array's device address (cudaGetSymbolAddress) with that device current; make
 * that first call before any stream capture.  The address is cached per device and
 * looked up again when the device's context has changed (a device reset reloads the
 * library's module; call again before capturing after a reset).  Every call on a
 * device shares the array
 * and leaves its contents behind: calls whose work overlaps on the GPU (other streams,
 * other threads) race on it and must be serialised by the caller. */
srmra_status srmra_loglik_noalloc(const float* y_dev, int64_t N, int32_t L, int32_t K,
                                  double sigma, const float* x_dev, const double* rho1_dev,
                                  const double* rho2_dev, double* lse_dev, double* ll_dev,
                                  void* cuda_stream);

/* Size in bytes of the fixed device array used by srmra_loglik_noalloc. */
int64_t srmra_noalloc_scratch_bytes(void);

/* Message of the last failing srmra_loglik_noalloc call in this thread. */
const char* srmra_noalloc_last_error(void);

/* srmra_sync -- wait for all work enqueued by this context. */
srmra_status srmra_sync(srmra_ctx* ctx);

/* srmra_destroy -- free the context and its device memory (NULL is a no-op).  Waits
 * for the context's pending work first. */
void srmra_destroy(srmra_ctx* ctx);

/* srmra_last_error -- message of the last failing call on ctx (ctx may be NULL: then
 * the message of the last failing srmra_create in this thread). */
const char* srmra_last_error(const srmra_ctx* ctx);

/* srmra_version -- library version string. */
const char* srmra_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SRMRA_H */
