/*
 * fairrank.h -- C ABI of libfairrank: NSW fair ranking by gradient ascent over batched Sinkhorn
 * solves on one GB300 (sm_103a).
 *
 * Method: Uehara et al., "Fast solution to the fair ranking problem using the Sinkhorn algorithm"
 * (arXiv 2406.10262). Each consumer u gets a stochastic ranking X_u (|I| items x m columns) that
 * satisfies Eqs. (1)-(3): every item row sums to 1, each of the K real slots receives mass 1, and
 * a last dummy slot receives |I|-K (Sec. 2; it is dropped when |I| == K). The library maximises
 * the Nash social welfare F = sum_i log Imp_i (Eq. 5), Imp_i = sum_u sum_{k<K} r(u,i) e(k) x_uik
 * (Eq. 4), over transport costs C (Problem (8)): every step solves the entropic optimal-transport
 * problem (7) of every consumer by log-domain Sinkhorn, reduces impacts across consumers, and
 * moves C along grad_C F(X*(C)) with Adam (Algorithm 1, Sec. 4.1).
 *
 * Conventions for every entry point:
 *  - Return value: FR_OK or an error status; fr_last_error() gives a message. Nothing throws.
 *  - Pointers flagged `on_device` are device pointers (e.g. torch CUDA tensors) used on the
 *    context's stream; other pointers are host memory. The library copies inputs, owns all device
 *    state it allocates (cudaMalloc in fr_create / fr_set_relevance) and frees it in fr_destroy.
 *    Outputs go to caller buffers of the stated size.
 *  - Layouts are row-major and dense: relevance [n_users][n_items], policy / costs / moments
 *    [n_users][n_items][n_cols], column potentials [n_users][n_cols].
 *  - A context belongs to one host thread at a time; there is no global mutable state.
 *  - Every call is stream-ordered on the context's stream and returns after the results it
 *    reports are available on the host (host outputs) or enqueued (device outputs).
 */
#ifndef FAIRRANK_H
#define FAIRRANK_H
#include <stdint.h>

#if defined(__GNUC__)
#define FR_API __attribute__((visibility("default")))
#else
#define FR_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fr_ctx fr_ctx; /* opaque; owns all device state of one problem */

typedef enum {
    FR_OK = 0,
    FR_EINVAL = 1,    /* invalid argument or configuration (message says which) */
    FR_ENOMEM = 2,    /* device allocation failed */
    FR_ECUDA = 3,     /* a CUDA call failed (message carries cudaGetErrorString) */
    FR_ENUMERIC = 4,  /* an impact became non-positive or a value non-finite */
    FR_ETIMEOUT = 5,  /* a bounded device-side wait expired */
    FR_ESTATE = 6,    /* call order: e.g. fr_step before fr_set_relevance / fr_set_exposure */
    FR_EUNSUPPORTED = 7 /* shape outside the compiled kernel variants (message gives the limit) */
} fr_status;

enum { FR_PARAM_FULL_C = 0, /* free cost tensor C of Problem (8) (the paper's parametrisation) */
       FR_PARAM_ITEM = 1 }; /* c_uik = -r(u,i) e(k) exp(theta_i): per-item variables theta */
enum { FR_GRAD_IMPLICIT = 0, FR_GRAD_UNROLLED = 1 };
enum { FR_ADAM = 0, FR_SGD = 1 };
enum { FR_F32 = 0, FR_BF16 = 1, FR_F64 = 2 };

typedef struct fr_config {
    int32_t n_users, n_items, n_slots; /* |U|, |I|, K; requires 1 <= K <= |I| */
    int32_t param;          /* FR_PARAM_FULL_C | FR_PARAM_ITEM */
    double  epsilon;        /* entropic regularisation of Problem (7), > 0 */
    int32_t sinkhorn_iters; /* L >= 1 Sinkhorn iterations per consumer per step */
    int32_t warm_start;     /* 1: each solve starts from the previous solve's column potentials */
    int32_t grad_mode;      /* FR_GRAD_IMPLICIT: differentiates the optimality conditions of
                               Problem (7) at the emitted policy. FR_GRAD_UNROLLED: the exact
                               derivative of the L-iteration Sinkhorn map that produced the policy
                               (reverse sweep over the iterations, the warm start held constant);
                               FR_PARAM_ITEM needs n_items <= 6144 (2048 unless n_cols is 6, 11 or
                               21), FR_PARAM_FULL_C (dL/dc for every cell) n_cols <= 32 and
                               n_items <= 1024 (n_cols <= 16) or 512, else FR_EUNSUPPORTED */
    int32_t ckpt_every;     /* FR_GRAD_UNROLLED: every ckpt_every-th iterate of the column
                               potentials is stored per consumer (ceil(L / ckpt_every) n_cols
                               floats); the rest are recomputed. With 1 and FR_PARAM_ITEM each
                               iteration's column sums are kept too (L n_cols more floats per
                               consumer) and the adjoint does no forward re-runs. >= 1 */
    int32_t optimizer;      /* FR_ADAM (PyTorch Adam, maximize) | FR_SGD */
    double  lr, beta1, beta2, adam_eps;
    int32_t rel_dtype;      /* storage of r on the device: FR_F32 | FR_BF16 */
    int32_t max_wait_polls; /* polls a bounded device-side wait makes (the wait of a kernel for its
                               staged bulk copies, and of the envy contraction for its tensor-core
                               work) before it gives up: the kernel then records FR_ETIMEOUT, waits
                               for its own copies in flight with the default bound and stops, so
                               the CUDA context stays usable. 0: the default (2^26 polls, many
                               seconds); -1: no poll at all, every such wait expires at once (for
                               testing the failure path); other negative values: FR_EINVAL */
    int32_t reserved[6];    /* must be zero */
} fr_config;

/* Fills cfg with the defaults: epsilon 1, L = 50, warm start, implicit gradient, checkpoint every
   10, Adam with lr 0.1 (FR_PARAM_FULL_C) or 0.05 (FR_PARAM_ITEM), betas (0.9, 0.999), eps 1e-8,
   FP32 relevance. Algorithm 1 leaves these values open; they are this library's choices. */
FR_API void fr_config_default(fr_config* cfg, int32_t n_users, int32_t n_items, int32_t n_slots,
                       int32_t param);

/* Number of stored columns m: n_slots + 1 when n_items > n_slots (dummy slot of Sec. 2), else
   n_slots. */
FR_API int32_t fr_num_cols(int32_t n_items, int32_t n_slots);

/* Creates a context on the current CUDA device. stream: a cudaStream_t (NULL = legacy default
   stream); every later call is ordered on it. Allocates the optimiser state (zero costs / theta =
   the uniform policy, Algorithm 1's unspecified initialisation). FR_EINVAL on a bad config,
   FR_EUNSUPPORTED on a shape outside the compiled variants, FR_ENOMEM. *out is NULL on error.
   Largest n_items by n_cols (a CTA has at most 512 threads and 227 KB of shared memory):
   FR_PARAM_FULL_C 4096 for 11 columns, 2048 for 2-16 and 21, 1024 for 17-24 (except 21), from
   992 down to 776 for 25-32, 512 for 33-45, from 496 down to 320 for 46-64;
   FR_PARAM_ITEM 12288 for 6, 11 or 21 columns with BF16 relevance (11400, 11352 and 11088 with
   FP32), 4096 for the other counts up to 32. */
FR_API fr_status fr_create(const fr_config* cfg, void* stream, fr_ctx** out);
FR_API fr_status fr_destroy(fr_ctx* ctx);

/* Resets the optimiser state to its initial value (costs / theta 0, moments 0, potentials 0,
   t = 0) on the device without host transfers; the policy becomes stale. */
FR_API fr_status fr_reset(fr_ctx* ctx);

/* Relevance r(u,i) of Eq. (4): n_users x n_items, row stride ld elements (>= n_items), dtype
   FR_F32 | FR_F64 | FR_BF16 (raw bfloat16 bits). Values must be finite and >= 0 and every item
   needs some r(u,i) > 0 (log Imp_i of Eq. 5), else FR_EINVAL. Copied (and converted to the
   configured storage dtype). */
FR_API fr_status fr_set_relevance(fr_ctx* ctx, const void* r, int32_t dtype, int64_t ld,
                           int32_t on_device);

/* Exposure e(k) of the K real slots (Eq. 4), host doubles, each > 0 and finite (FR_EINVAL), K must
   equal cfg.n_slots. The dummy slot has exposure 0. The certificate of fr_certificate additionally
   needs e non-increasing. Copied. */
FR_API fr_status fr_set_exposure(fr_ctx* ctx, const double* e, int32_t K);

/* n_steps >= 0 ascent steps of Algorithm 1. If the policy is stale (first call, or after
   fr_set_*), first solves Sinkhorn for the current parameters. Each step: gradient of F at the
   current policy, optimiser update, Sinkhorn for every consumer with the new parameters, impacts
   and F (FP64). nsw_trace (host, nullable, n_steps doubles) receives F after each step.
   FR_ESTATE before both fr_set_relevance and fr_set_exposure; FR_ENUMERIC if an impact became
   non-positive or non-finite (the state is then undefined). */
FR_API fr_status fr_step(fr_ctx* ctx, int32_t n_steps, double* nsw_trace);

/* Algorithm 1 with threshold t on ||grad F||_2 (gradient with respect to the optimised variable):
   runs steps until one whose gradient norm is <= t (that step's update is applied) or max_steps.
   *steps_done and *nsw_out (nullable) report the steps run and the final F. The loop runs on the
   device: one CUDA graph launch whose conditional while node repeats chunks of steps until the
   stop flag raised by the FP64 reduction, with no host round trip per step or chunk. */
FR_API fr_status fr_solve(fr_ctx* ctx, double t, int32_t max_steps, int32_t* steps_done,
                   double* nsw_out);

/* Per-step record of the last fr_step or fr_solve call (host doubles, each nullable, the first
   min(n, recorded) steps): nsw[k] = F after step k (FP64), grad_norm[k] = ||grad F||_2 of step k
   (FP64, the norm Algorithm 1's stop test compares with t, taken at the policy before that step's
   update). *n_steps (nullable) receives the number of steps recorded. FR_EINVAL if n < 0. */
FR_API fr_status fr_trace(fr_ctx* ctx, int32_t n, double* nsw, double* grad_norm, int32_t* n_steps);

/* Current impacts Imp_i (Eq. 4; host, n_items doubles, nullable), user utility sum_i Imp_i / |U|
   (Sec. 4.1, nullable) and F (Eq. 5, nullable) of the current policy; solves first if stale. */
FR_API fr_status fr_impacts(fr_ctx* ctx, double* imp_out, double* utility_out, double* nsw_out);

/* Policy X_u of consumers u0 .. u0+n_u-1 (rows of Eqs. (1)-(3)): float [n_u][n_items][n_cols],
   host or device (on_device). Rows sum to 1 to rounding; the column residual is the remaining
   Sinkhorn error. FR_EINVAL if the range leaves [0, n_users). */
FR_API fr_status fr_policy(fr_ctx* ctx, int32_t u0, int32_t n_u, float* x_out, int32_t on_device);

/* Gradient at the current policy of L = sum_i omega_i Imp_i, omega (n_items floats, nullable;
   NULL means omega_i = 1/Imp_i, i.e. L = F of Eq. 5) in the configured grad_mode. dparam:
   FR_PARAM_FULL_C dL/dC [n_users][n_items][n_cols]; FR_PARAM_ITEM dL/dtheta [n_items]. dr
   (nullable): dL/dr [n_users][n_items]. All pointers host or device per on_device. */
FR_API fr_status fr_grad(fr_ctx* ctx, const float* omega, float* dparam, float* dr, int32_t on_device);

/* Optimiser state: parameters (FR_PARAM_FULL_C: C [n_users][n_items][n_cols]; FR_PARAM_ITEM:
   theta [n_items]), Adam moments (same shape), column potentials g [n_users][n_cols] in the units
   of C (the warm start of the next solve) and the Adam step count t. Any pointer may be NULL to
   leave that part unchanged (set) or unread (get). Setting marks the policy stale. */
FR_API fr_status fr_set_state(fr_ctx* ctx, const float* param, const float* m1, const float* m2,
                       const float* g, int64_t t, int32_t on_device);
FR_API fr_status fr_get_state(fr_ctx* ctx, float* param, float* m1, float* m2, float* g, int64_t* t,
                       int32_t on_device);

/* Evaluation metrics of Sec. 4.1 at the current policy (host doubles, each nullable): user
   utility, mean max envy (1/|I|) sum_i max_j (Imp_i(X_j) - Imp_i(X_i)), and the percentage of
   items whose impact is more than 10% above / below that of the uniform policy x_uik = b_k/|I|.
   Imp_i(X_j) = sum_u r(u,i) sum_{k<K} e_k x_ujk is formed on the tensor cores from three TF32
   products per term (hi*hi + hi*lo + lo*hi of each operand's TF32 split), accumulated in FP32: the
   error is that of an FP32 contraction. Needs about n_users x n_items x 20 bytes of scratch (V and
   the TF32 planes of R and V; allocated on first use). FR_ETIMEOUT if a bounded device wait of the
   contraction expired. */
FR_API fr_status fr_metrics(fr_ctx* ctx, double* utility, double* mean_envy, double* better_pct,
                     double* worse_pct);

/* Per-item envy of Sec. 4.1 at the current policy: envy[i] = max_j (Imp_i(X_j) - Imp_i(X_i)) for
   every item, host doubles [n_items] (non-NULL, else FR_EINVAL). The same contraction and error as
   fr_metrics, whose mean envy is the mean of this vector; same scratch and FR_ETIMEOUT. */
FR_API fr_status fr_item_envy(fr_ctx* ctx, double* envy);

/* Optimality certificate of the current policy (host doubles, each nullable). F is concave in X
   and each X_u ranges over the polytope of Eqs. (1)-(3), so F* - F(X) <= max_Y <grad F(X), Y - X>;
   with e non-increasing the maximising Y_u ranks the items by r(u,i)/Imp_i (rearrangement), giving
   gap = sum_u [sum_{k<K} e_k (k-th largest r(u,i)/Imp_i) - sum_{i,k<K} (r(u,i)/Imp_i) e_k x_uik].
   The bound holds for exactly feasible X; the emitted X has exact rows and a column residual
   max_{u,k} |sum_i x_uik - b_k|, reported beside it. Needs e non-increasing for the bound. */
FR_API fr_status fr_certificate(fr_ctx* ctx, double* gap, double* col_residual);

/* Replaces ctx's max_wait_polls (see fr_config; 0 restores the default). After an FR_ETIMEOUT the
   optimiser state is undefined: fr_reset, or fr_set_state, brings the context back to a defined
   state. FR_EINVAL for a value below -1. */
FR_API fr_status fr_set_wait_limit(fr_ctx* ctx, int32_t max_wait_polls);

/* Message of the last failing call on ctx (or of the last failing fr_create on this thread when
   ctx is NULL). Valid until the next call on ctx. */
FR_API const char* fr_last_error(const fr_ctx* ctx);

/* ---- batched markets ---------------------------------------------------------------------- */

/* Many independent instances of Problem (8) (each market its own consumers, items, slots,
   relevance, exposure and parameters), advanced together. FR_PARAM_ITEM: per ascent step one
   gradient and one Sinkhorn launch per kernel shape (concurrent), one theta update and one impact
   reduction over all markets. FR_PARAM_FULL_C (free costs, the paper's parametrisation): per ascent
   step one launch of the fused gradient + Adam + Sinkhorn kernel per kernel shape (concurrent) and
   one impact reduction over all markets. Chunks of steps are replayed as a CUDA graph. Results
   equal those of one FairRank context per market (same per-consumer arithmetic). The paper runs
   Algorithm 1 on one market at a time; batching is this library's packaging for many small
   markets on one GPU. */
typedef struct fr_batch fr_batch; /* opaque; owns all device state of the markets */

/* cfgs[0 .. n_markets): all FR_PARAM_ITEM (n_cols <= 32, n_items <= 4096) or all FR_PARAM_FULL_C
   (FP32 relevance, the single-market limits of fr_create), each FR_GRAD_IMPLICIT; every field except
   n_users, n_items and n_slots must equal cfgs[0]'s (FR_EINVAL). stream: as fr_create. */
FR_API fr_status fr_batch_create(const fr_config* cfgs, int32_t n_markets, void* stream,
                                 fr_batch** out);
FR_API fr_status fr_batch_destroy(fr_batch* b);
/* theta, moments, potentials and step state of every market back to their initial values. */
FR_API fr_status fr_batch_reset(fr_batch* b);
/* As fr_set_relevance / fr_set_exposure for one market (0 <= market < n_markets). */
FR_API fr_status fr_batch_set_relevance(fr_batch* b, int32_t market, const void* r, int32_t dtype,
                                        int64_t ld, int32_t on_device);
FR_API fr_status fr_batch_set_exposure(fr_batch* b, int32_t market, const double* e, int32_t K);
/* Times, for every kernel shape, each candidate of rows per thread (8 / 16 / 24 where a kernel
   exists; free-cost shapes fix it) and consumers per chunk (4 / 16) with one Sinkhorn launch on the
   markets' own data and keeps the fastest. Runs by itself before the first solve; the warm-start
   potentials are kept. */
FR_API fr_status fr_batch_autotune(fr_batch* b);
/* n_steps >= 0 ascent steps of Algorithm 1 in every market (first solves every market if stale).
   nsw_trace (host, nullable): [n_steps][n_markets] doubles, F of each market after each step. */
FR_API fr_status fr_batch_step(fr_batch* b, int32_t n_steps, double* nsw_trace);
/* As fr_impacts / fr_policy for one market. */
FR_API fr_status fr_batch_impacts(fr_batch* b, int32_t market, double* imp_out, double* utility_out,
                                  double* nsw_out);
FR_API fr_status fr_batch_policy(fr_batch* b, int32_t market, int32_t u0, int32_t n_u, float* x_out,
                                 int32_t on_device);
/* theta of one market (host, n_items floats); FR_EINVAL for free-cost markets. */
FR_API fr_status fr_batch_get_theta(fr_batch* b, int32_t market, float* theta_out);
/* Kernel shapes and the autotuner's choices: *n_buckets shapes; table (nullable, cap rows of 6
   int32): kernel columns, markets, largest n_items, rows per thread, CTA threads, consumers per
   chunk. */
FR_API fr_status fr_batch_tuning(const fr_batch* b, int32_t* n_buckets, int32_t* table, int32_t cap);
/* Message of the last failing call on b (or of the last failing fr_batch_create on this thread
   when b is NULL). */
FR_API const char* fr_batch_last_error(const fr_batch* b);
/* Kernels launched on b since creation (graph replays count their kernels). */
FR_API int64_t fr_batch_launch_count(const fr_batch* b);

/* ---- measurement helpers --------------------------------------------------------------- */

/* Number of kernels the library launched on ctx since creation (every launch is counted on the
   host when it is enqueued, graph replays count their kernels). */
FR_API int64_t fr_launch_count(const fr_ctx* ctx);

/* Times the kernels of the ascent step with CUDA events recorded on the library stream around
   each launch: runs n_steps >= 1 steps with direct launches (no graph) and writes mean durations
   in milliseconds. FR_PARAM_FULL_C: the fused gradient+Adam+Sinkhorn kernel (ms[0]), the
   cross-consumer reduction kernel (ms[1]) and a Sinkhorn-only solve of the same costs (ms[2],
   launched after each step). FR_PARAM_ITEM: the Sinkhorn kernel (ms[0]), the reduction kernel
   (ms[1]) and the gradient kernel (implicit or adjoint) plus the theta update (ms[2]).
   FR_PARAM_FULL_C with FR_GRAD_UNROLLED: the Sinkhorn kernel (ms[0]), the reduction (ms[1]) and
   the adjoint kernel with the optimiser step on C (ms[2]). Advances the optimiser state like
   fr_step. */
FR_API fr_status fr_time_kernels(fr_ctx* ctx, int32_t n_steps, double* ms);

/* The compiled kernel variant that serves ctx's Sinkhorn sweep (diagnostics, e.g. to name the
   kernel a profile refers to): out[0] column bucket, out[1] rows per thread, out[2] 1 if compiled
   for exactly n_cols columns, out[3] CTA size, out[4] shared-tile column stride in floats of the
   free-cost tile sweep (0: costs held in registers; always 0 for FR_PARAM_ITEM), out[5] persistent
   grid size. FR_EINVAL if ctx or out is NULL. */
FR_API fr_status fr_kernel_variant(const fr_ctx* ctx, int32_t* out);

/* Diagnostics of the free-cost Sinkhorn sweeps: writes the number of consumer solves since the
   last fr_reset that left the sweep's exponential form (the row-shifted kernel 2^(g'_k - c~_ik)
   held in shared memory or registers, one multiply per cell) for its log form (one exp2 per
   cell), because a column potential drifted more than 30 log2 units from its value at the start
   of the solve. Warm-started ascent steps stay in the exponential form; cold starts from widely
   spread costs leave it. Kernels with the exponential form: the tile sweep (out[4] of
   fr_kernel_variant > 0) and the register sweep of at most 11 columns; the wider register sweeps
   and FR_PARAM_ITEM always report 0. Synchronises with ctx's work. FR_EINVAL if ctx or out is
   NULL. */
FR_API fr_status fr_sweep_stats(fr_ctx* ctx, int64_t* log_form_solves);

/* Measures the sustained rate of ex2.approx.f32 on the current device with a dependent-chain-free
   microbenchmark (grid = SMs x 4 CTAs): writes exp2 evaluations per second. Used as the measured
   denominator of the Sinkhorn roofline. */
FR_API fr_status fr_measure_ex2_rate(double* ex2_per_second);

/* Measures the on-chip rates that bound the Sinkhorn sweeps on the current device (each probe one
   launch of SMs x 4 or 8 CTAs, timed with CUDA events after a warm-up launch) and writes the first
   n of: out[0] ex2.approx.f32 results per second; out[1] shared-memory load bandwidth in bytes per
   second with 8-byte loads and out[2] with 16-byte loads (consecutive lanes, conflict-free: the
   sweeps' access pattern); out[3] FP32 fused multiply-adds per second (scalar fma.rn.f32) and
   out[4] with packed fma.rn.f32x2 (two per instruction); out[5] the SM clock in MHz during the
   probes (clock64 cycles over global-timer nanoseconds, median of the probes). These are the
   measured denominators of the rooflines the benchmark reports. 1 <= n <= 6, else FR_EINVAL. */
FR_API fr_status fr_measure_peaks(double* out, int32_t n);

/* Self-check of the logarithm in the Sinkhorn column updates: log2_near1(y) evaluates log2 for
   |y - 1| < 2^-5 as the Taylor series of ln(1 + t) / ln 2 (t = y - 1, coefficients +-1/(n ln 2)
   through t^6) and calls log2f elsewhere. Evaluates it on the device for every float y in that
   range and writes out[0] its largest relative error against log2 in double precision, out[1] the
   same for log2f(y), out[2] the number of values at y = 1 that were not exactly 0. FR_EINVAL if
   out is NULL. */
FR_API fr_status fr_check_log2_near1(double* out);

/* ---- allocation-free evaluation --------------------------------------------------------- */

/* For callers that cannot allocate device memory. The paper has no counterpart to this entry
   point: it packages the library's Sinkhorn solve and impact reduction for code whose device
   memory belongs to someone else -- a framework's caching allocator or a fixed arena that must not
   grow -- and for latency-critical loops in which cudaMalloc / cudaFree, which can synchronize the
   whole device, must not be called. It never calls cudaMalloc, cudaFree or any allocating library
   routine.

   Computes what fr_impacts reports for a context created with warm_start = 0 whose costs are C:
   sinkhorn_iters iterations of every consumer's solve from zero column potentials, the impacts
   Imp_i and F = sum_i log Imp_i.
   Inputs (device memory, 16-byte aligned): C float [n_users][n_cols][ld], slot-major within a
   consumer (C[(u*n_cols + k)*ld + i] = c_uik); r float [n_users][ld]; ld a multiple of 8 and
   >= n_items (entries beyond n_items are ignored). e: host doubles [n_slots], each > 0.
   Outputs (device memory): imp_out double [n_items]; nsw_util_out double [2] = {F, user utility}.
   F is -inf or NaN if an impact is not positive (no status is read back: the call stays
   asynchronous).
   Scratch: one static array of 8 MiB in device memory, which every GPU that loads the library
   keeps from load until process exit. The problem must fit in it: about 8 bytes per consumer and
   column plus 4 bytes per item and CTA (the CTA count shrinks to fit); larger problems return
   FR_EUNSUPPORTED with a message in fr_last_error(NULL), as do shapes outside the compiled kernel
   variants. The first call on each device looks up the array's device address
   (cudaGetSymbolAddress, with that device current); make that first call before any stream
   capture. Work is enqueued on `stream` (NULL = legacy default stream). Every call uses the same
   array and leaves its contents behind: calls that can overlap on the GPU (other streams, other
   host threads) race with each other and corrupt each other's results. */
FR_API fr_status fr_nsw_eval_noalloc(const float* C, const float* r, int64_t ld, const double* e,
                                     int32_t n_users, int32_t n_items, int32_t n_slots,
                                     double epsilon, int32_t sinkhorn_iters, double* imp_out,
                                     double* nsw_util_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif
