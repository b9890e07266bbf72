/*
 * pl.h -- C ABI of the GB300 (sm_103a) library for Monte Carlo
 * Kolmogorov-Smirnov cutoffs of the discrete power law with a
 * maximum-likelihood exponent (Rappos & Robert, "Using GPU Simulation to
 * Accurately Fit to the Power-Law Distribution", 2013).
 *
 * The law (Eq. 1, with a lower end xmin; the paper's case is xmin = 1):
 *     p(k) = k^-alpha / zeta(alpha, xmin),   k = xmin, xmin+1, ...,  alpha > 1.
 * The fit (Eq. 2):   zeta'(alpha, xmin) / zeta(alpha, xmin) = -(1/n) sum ln x_i.
 * The statistic (Eq. 3):   D = sup_x |F(x) - S(x)|, F the law at the fitted
 * exponent, S the empirical CDF.
 * Cutoffs (Section 3): quantiles of D over replicates simulated at (alpha, n).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Memory: the caller owns every buffer.  Pointers documented "device" must
 *   be device (or managed) memory of the context's GPU; "host" pointers are
 *   ordinary host memory.  The library allocates only its own workspace,
 *   inside the byte budget given to pl_create, and returns PL_ENOMEM rather
 *   than exceed it.
 * - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *   Work is stream ordered.  Entry points with a host output synchronise
 *   that stream before returning; the others return once the work is
 *   enqueued.  One context must not be used from two streams at once (its
 *   workspace is shared); create one context per concurrent stream.
 * - Errors: every entry point returns a pl_status; nothing throws or aborts
 *   across the ABI.  pl_last_error gives a one-line description of the last
 *   failure on that context.  Errors found on the device (a bounded wait that
 *   ran out, bad data values) are latched in the context and reported by the
 *   next pl_sync or by the next entry point with a host output.
 * - Randomness: draw i of replicate r is a pure function of
 *   (seed, cell_id, r, purpose, i) through Philox4x32-10 (key = seed): the
 *   high 32 of its 53 bits are word i mod 4 of the block with counter
 *   (i/4, r, cell_id, purpose), the low 21 the top bits of the same word of
 *   the block with counter (i/4, r, cell_id, purpose + 2^31), which the
 *   samplers generate only when a draw needs them.  Sampled values never depend on
 *   launch shape, batching, the warp/block split or the precision form; for a
 *   given split and precision form every result is bit-identical whether a
 *   cell runs alone or with others.  Changing the split changes the rounding
 *   of alpha-hat and D at the 1e-15 level.  purpose (< 2^31): 0 = cutoff
 *   simulation, 1 = parametric bootstrap, 2 = test data.
 * - Heavy tail: simulated values are uint64 and saturate at 2^62.
 */
#ifndef PL_H_
#define PL_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pl_ctx pl_ctx;

typedef enum {
  PL_OK = 0,
  PL_EINVAL = 1,   /* an argument is out of its domain */
  PL_ENOMEM = 2,   /* workspace would exceed the context's byte budget */
  PL_ENOCONV = 3,  /* a Newton solve hit its iteration cap */
  PL_ETIMEOUT = 4, /* a bounded device wait ran out */
  PL_ECUDA = 5,    /* a CUDA runtime call failed */
  PL_EBUSY = 6     /* reserved */
} pl_status;

typedef enum {
  PL_FP64 = 0,      /* every floating-point step in binary64 */
  PL_FP32_BULK = 1  /* log-sums, CDF prefix sums and D comparisons in binary32
                       with compensated accumulation; Hurwitz zeta, Newton solve
                       and normaliser stay binary64 */
} pl_precision;

/* One cell of a cutoff table: `replicates` samples of size n from the law at
 * (alpha, xmin); cell_id (< 2^32) keys its random streams. */
typedef struct {
  double alpha;
  uint64_t xmin;
  int64_t n;
  int64_t replicates;
  uint64_t cell_id;
} pl_cell;

/* Create a context on CUDA device `device`; the library's workspace never
 * exceeds mem_budget_bytes (0 = 40 GiB).  Besides the workspace, the context
 * keeps the fit tables (Eq. 2's exponent as a function of the mean log, a
 * function of xmin alone) of the first 16 values of xmin its calls use, about
 * 0.2 MB each, and later calls copy them on the device instead of building
 * them again.  *out receives the context.
 * Errors: PL_EINVAL (out NULL, bad device), PL_ECUDA. */
pl_status pl_create(pl_ctx **out, int device, size_t mem_budget_bytes);

/* Free the context and its workspace (synchronises the device first). */
void pl_destroy(pl_ctx *ctx);

/* Text of the last error on ctx ("" if none).  Owned by the context. */
const char *pl_last_error(const pl_ctx *ctx);

/* Synchronise `stream` and report device-side errors latched since the last
 * report (PL_ETIMEOUT, PL_EINVAL for bad data values, PL_ECUDA). */
pl_status pl_sync(pl_ctx *ctx, void *stream);

/* Counters accumulated on the device since pl_create (diagnostics; no
 * counterpart in the paper). */
typedef struct {
  uint64_t newton_capped;  /* Newton solves that hit the iteration cap */
  uint64_t tail_draws;     /* draws inverted in binary64 beyond the threshold table */
  uint64_t global_sorts;   /* replicates with more than 512 values beyond the
                              dense histogram (large spill sorts) */
  uint64_t fit_fallbacks;  /* fits by the full Newton iteration instead of the
                              one-step polish from the interpolated start */
  uint64_t resampled;      /* replicates drawn a second time because their
                              record's spill slot overflowed */
} pl_counter_info;

/* Synchronises `stream` and copies the counters to *out (host). */
pl_status pl_counters(pl_ctx *ctx, void *stream, pl_counter_info *out);

/* Issue rates of the units that bound the kernels, measured on the
 * context's GPU (not a step of the method; the paper has no counterpart):
 * each probe kernel keeps one 1024-thread block per SM busy with eight
 * independent chains of one instruction, and the longest block's clock64
 * count over the CUDA-event time gives the SM clock of the run.  The samplers' ceiling
 * is the 32x32->64-bit multiply (Philox4x32-10 takes five per 32-bit draw);
 * the fit and the binary64 KS run on the binary64 pipe.  Takes a few
 * milliseconds; uses the context's workspace (about 600 KB per 100 SMs).
 * Synchronises `stream`.  Errors: PL_EINVAL (null out), PL_ENOMEM, PL_ECUDA. */
typedef struct {
  double sm_clock_mhz;         /* SM clock during the multiply probe */
  double mul_wide_per_sm_clk;  /* mul.wide.u32 per SM per clock */
  double lop3_per_sm_clk;      /* three-input logic operations per SM per clock */
  double dfma_per_sm_clk;      /* binary64 fused multiply-adds per SM per clock */
  double philox_words_per_s;   /* 32-bit Philox4x32-10 words per second, whole GPU */
  int32_t sms;                 /* SMs of the GPU */
  int32_t pad;
} pl_probe_info;
pl_status pl_probe_rates(pl_ctx *ctx, void *stream, pl_probe_info *out);

/* Tracing (no counterpart in the paper, which times whole runs with clock()).
 * With tracing on, pl_ks_cutoffs and pl_bootstrap_pvalue record CUDA events
 * on their stream around each phase; pl_trace synchronises `stream` and
 * returns the durations of the last traced call and the number of kernels
 * this context has launched since pl_create. */
typedef struct {
  uint64_t launches;   /* kernels launched by this context */
  float law_ms;        /* last traced call: law-table set-up kernels */
  float replicate_ms;  /* last traced call: all replicate kernels (every wave) */
  float select_ms;     /* last traced call: quantile selection / p count */
  float total_ms;      /* last traced call: first to last phase */
  float sample_ms;     /* last traced call: sampler launches, summed over waves */
  float finish_ms;     /* last traced call: finisher launches, summed over waves */
  uint32_t waves;      /* last traced call: number of waves */
  uint64_t draws;      /* last traced call: draws simulated */
  uint32_t sample_launches; /* last traced call: sampler kernel launches (one
                               per wave, form and binning mode) */
} pl_trace_info;

pl_status pl_set_tracing(pl_ctx *ctx, int on);
pl_status pl_trace(pl_ctx *ctx, void *stream, pl_trace_info *out);

/* Draws from the law (Eq. 1 with lower end xmin) by inverse CDF: with
 * v = m 2^-53 in (0, 1], X = min{k >= xmin : P(X > k) < v}.
 * Writes nrep * n values, row r (replicate rep0 + r) at out_dev[r * n].
 * out_dev: device, uint64[nrep * n].  Errors: PL_EINVAL (alpha <= 1,
 * xmin < 1, n < 1, nrep < 1, cell_id >= 2^32, rep0 + nrep > 2^32,
 * n > 2^34, purpose >= 2^31). */
pl_status pl_sample(pl_ctx *ctx, double alpha, uint64_t xmin, uint64_t seed,
                    uint64_t cell_id, uint32_t purpose, uint64_t rep0,
                    int64_t nrep, int64_t n, uint64_t *out_dev, void *stream);

/* Maximum-likelihood exponent of a data set (Eq. 2).  If every value equals
 * xmin the log-sum is increased by ln((xmin+1)/xmin) (one point counted as
 * xmin+1), as the paper's code does for xmin = 1.  x_dev: device, int32[n],
 * every value >= xmin.  alpha_hat_host: host double.  Synchronises `stream`.
 * Errors: PL_EINVAL (n < 1, n > 2^31 - 1, xmin < 1, xmin > 2^31, a value
 * < xmin), PL_ENOCONV. */
pl_status pl_fit_mle(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                     uint64_t xmin, double *alpha_hat_host, void *stream);

/* KS distance (Eq. 3) between the empirical CDF of x and the law at
 * exponent alpha (alpha > 1; pass the fitted exponent to use the paper's
 * tables).  x_dev: device, int32[n] (1 <= n <= 2^31 - 1), values >= xmin.
 * D_host: host double.  Synchronises `stream`.  Errors: PL_EINVAL. */
pl_status pl_ks_stat(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                     uint64_t xmin, double alpha, pl_precision prec,
                     double *D_host, void *stream);

/* Cutoff table (Section 3, Table 1): for every cell simulate `replicates`
 * samples of size n at (alpha, xmin) (purpose 0), fit each by maximum
 * likelihood, compute its D at the fitted exponent, and return the order
 * statistics D_(i), i = floor(R q_j) (0-based, clamped to R-1), for the nq
 * quantiles q_j in (0, 1).
 * cells: host, pl_cell[ncells].  q: host, double[nq].
 * cutoffs: device or host, double[ncells * nq] (row per cell); a host
 *   pointer makes the call synchronise `stream`.
 * D_dev_opt: NULL or device, per-replicate D of every cell concatenated in
 *   cell order (double for PL_FP64, float for PL_FP32_BULK).
 * alpha_hat_dev_opt: NULL or device double, per-replicate fitted exponents,
 *   same layout.
 * Errors: PL_EINVAL (ncells < 1, nq < 1, q outside (0,1), alpha <= 1,
 * xmin < 1, n < 1, replicates < 1, cell_id >= 2^32), PL_ENOMEM. */
pl_status pl_ks_cutoffs(pl_ctx *ctx, const pl_cell *cells, int ncells,
                        uint64_t seed, const double *q, int nq,
                        pl_precision prec, double *cutoffs, void *D_dev_opt,
                        double *alpha_hat_dev_opt, void *stream);

/* Cutoff table with the multinomial histogram sampler (a large-n variant;
 * not in the paper): each replicate's histogram is drawn by conditional
 * binomials on the inverse-CDF sampler's law, through its integer thresholds
 * T (with T[-1] = 2^53 + 1, the index range [l, r) has mass
 * (T[l-1] - T[r-1]) 2^-53).  With B = 2048: the count beyond the first B
 * values is Bin(n, (T[B-1] - 1) 2^-53); the rest sits at node 1 of a binary
 * tree over [0, B), and node k of range [l, r) passes
 * Bin(c_k, (T[l-1] - T[mid-1]) / (T[l-1] - T[r-1])) of its count c_k to its
 * left child 2k (range [l, mid)) and the others to 2k + 1; leaves B .. 2B - 1
 * are the values xmin .. xmin + B - 1.  The values beyond are drawn one by
 * one as the inverse CDF of m' uniform on [1, T[B-1] - 1] (the high 64 bits
 * of a 64-bit random word times T[B-1] - 1, plus one).  The work grows with
 * the occupied values rather than with n (~780 binomials and ~780 single
 * values at alpha = 2, n = 10^6).  Random words (purpose 3): word j is 64
 * bits, the low half word 2 (j mod 2) and the high half word 2 (j mod 2) + 1
 * of the Philox block with counter (floor(j/2), replicate, cell_id, 3); a
 * binomial takes the uniform (top 53 bits + 1) 2^-53 of its word.  Word 0
 * is the count beyond, word k node k, word 2B + t the t-th value beyond.
 * Same law as pl_ks_cutoffs, a
 * different random stream, so results agree with pl_ks_cutoffs in
 * distribution, not value by value.  Arguments, outputs and errors as
 * pl_ks_cutoffs (every cell runs in the block form, n <= 2^21). */
pl_status pl_ks_cutoffs_multinomial(pl_ctx *ctx, const pl_cell *cells,
                                    int ncells, uint64_t seed, const double *q,
                                    int nq, pl_precision prec, double *cutoffs,
                                    void *D_dev_opt, double *alpha_hat_dev_opt,
                                    void *stream);

/* Autotuner of the warp/block split: replicates with n above the split use
 * the block-per-replicate form, the others the warp-per-replicate form.  The
 * split starts at 16384; pl_autotune times both forms on the context's GPU
 * (alpha = 2, 65,536 replicates, n = 2^9 .. 2^16) and sets the split to the
 * largest n bucket up to which the warp form is faster (at least 256).  The
 * split changes only rounding (see Randomness above).  Synchronises `stream`; *split_out (host, may be NULL) receives it.
 * pl_set_split sets it directly (1 <= split <= 65535). */
pl_status pl_autotune(pl_ctx *ctx, void *stream, int64_t *split_out);
pl_status pl_set_split(pl_ctx *ctx, int64_t split);

/* The tile settings of a context's simulations (not a step of the method;
 * the paper has no counterpart).
 * split: warp/block split as above.  item_reps: warp-form replicates per
 * work item (1..256; 0: sized by each plan, 256 or fewer when a simulation
 * is too small to give two items per resident sampler block).  hist_shift:
 * dense bins of a warp-form replicate, the smallest power of two >= 2n
 * (32..1024) times 2^hist_shift, kept within 32..1024; values beyond the dense
 * bins are spilled and sorted.  None of them changes sampled values; split
 * and hist_shift change the rounding of alpha-hat and D (1e-15 in the binary64
 * form, 1e-7 in the binary32-bulk form), item_reps changes nothing. */
typedef struct {
  int64_t split;
  int32_t item_reps;
  int32_t hist_shift;
  double best_ms;   /* pl_autotune_cells: the tuned call's time on the sample (ms) */
} pl_tuning;

/* Autotuner over the cells a caller will run: times pl_ks_cutoffs on the
 * same cells with at most sample_replicates replicates each (median of three
 * timed calls per setting) and picks, one after the other, the split (256,
 * 1,024, 4,096, 16,384, 65,535), the work-item size (32, 64, 128, 256; only
 * when the sample is the whole workload, as on a sample the plan's own item
 * sizing decides) and hist_shift (-1, 0, 1) that run fastest; leaves them set
 * on the context and
 * writes them to *out (host, may be NULL).  Synchronises `stream`.  On an
 * error the previous settings stay.  pl_set_tuning sets them directly.
 * Errors: PL_EINVAL, and those of pl_ks_cutoffs. */
pl_status pl_autotune_cells(pl_ctx *ctx, const pl_cell *cells, int ncells, pl_precision prec,
                            int64_t sample_replicates, pl_tuning *out, void *stream);
pl_status pl_set_tuning(pl_ctx *ctx, const pl_tuning *t);

/* The same computation split in two, so that the simulation can be enqueued
 * repeatedly (for example inside a captured CUDA graph).
 * pl_plan_cutoffs validates the cells (as pl_ks_cutoffs), allocates the
 * plan's own device memory (at most the context's byte budget), uploads its
 * cell, law and work tables, builds the law and fit tables on `stream`, and
 * synchronises `stream`.
 * pl_plan_run enqueues the simulation and the order statistics for `seed` on
 * `stream`: kernel launches and memsets only -- no allocation, no host
 * copy, no synchronisation.  cutoffs_dev: device double[ncells * nq];
 * D_dev_opt / alpha_hat_dev_opt as in pl_ks_cutoffs.  A plan uses its
 * context's counters: do not run it concurrently with other work of the
 * same context.
 * Errors: as pl_ks_cutoffs; PL_ENOMEM if the plan exceeds the budget. */
typedef struct pl_plan pl_plan;
pl_status pl_plan_cutoffs(pl_ctx *ctx, const pl_cell *cells, int ncells,
                          const double *q, int nq, pl_precision prec,
                          pl_plan **out, void *stream);
pl_status pl_plan_run(pl_plan *plan, uint64_t seed, double *cutoffs_dev,
                      void *D_dev_opt, double *alpha_hat_dev_opt, void *stream);
void pl_plan_destroy(pl_plan *plan);

/* Goodness of fit of a data set (Section 3's use of the tables, with the
 * bespoke cutoff computed by simulation): fit alpha-hat (Eq. 2), compute D
 * (Eq. 3), simulate B data sets of the same size at alpha-hat (purpose 1,
 * cell_id = request_id), refit each, and return p = #{D_b >= D} / B.
 * x_dev: device int32[n] (values >= xmin).  alpha_hat, D, p: host doubles.
 * Synchronises `stream`.  Errors: PL_EINVAL, PL_ENOMEM, PL_ENOCONV. */
pl_status pl_bootstrap_pvalue(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                              uint64_t xmin, int64_t B, uint64_t seed,
                              uint64_t request_id, pl_precision prec,
                              double *alpha_hat, double *D, double *p,
                              void *stream);

/* Serving engine: continuous batching of goodness-of-fit requests.  The
 * paper has no serving layer; each request computes what pl_bootstrap_pvalue
 * computes (Eq. 2, Eq. 3 and the bootstrap p-value at alpha-hat), and the
 * engine only schedules them.
 * `workers` host threads each own a context (with the fit tables of the
 * xmin values seen kept on the device) and a non-blocking stream, so up to `workers`
 * requests run on the GPU at the same time.  A request is admitted, oldest
 * first, when a worker is free and its planned device workspace (sized at a
 * fitted exponent of 1.4; each worker's context also keeps to the budget)
 * fits in mem_budget_bytes (0 = 40 GiB) beside the requests already running; a
 * request whose planned workspace exceeds the whole budget is not run: its
 * result (status PL_ENOMEM, NaN outputs) is ready at once.
 * Results are the same numbers pl_bootstrap_pvalue gives for that request
 * alone on a fresh context (seed, B, prec as given here; cell_id =
 * request_id), bit for bit.
 * pl_server_create: device as in pl_create; 1 <= workers <= 64; B >= 1.
 *   Errors: PL_EINVAL, PL_ECUDA, PL_ENOMEM.
 * pl_server_submit: x_host is host int32[n] (values >= xmin), copied before
 *   the call returns; request_id < 2^32.  Never blocks on the GPU.
 * pl_server_poll: moves up to max_results finished requests (host array
 *   pl_result[max_results]) in finishing order and returns their number,
 *   waiting up to wait_s seconds for the first one.
 * pl_server_now: seconds since create on the clock of the result times.
 * pl_server_load: queued requests, running requests, reserved bytes, and
 *   kernels launched by the finished requests (each pointer may be NULL).
 * pl_server_destroy: drops queued requests, waits for running ones, frees
 *   everything. */
typedef struct pl_server pl_server;
typedef struct {
  uint64_t request_id;
  int32_t status; /* pl_status of this request */
  int32_t pad;
  int64_t n;
  double alpha_hat, D, p;
  double submit_s, start_s, done_s; /* pl_server_now at submit, start, finish */
} pl_result;

pl_status pl_server_create(pl_server **out, int device, size_t mem_budget_bytes,
                           int workers, pl_precision prec, uint64_t seed,
                           int64_t B);
pl_status pl_server_submit(pl_server *srv, uint64_t request_id,
                           const int32_t *x_host, int64_t n, uint64_t xmin);
int pl_server_poll(pl_server *srv, pl_result *out, int max_results,
                   double wait_s);
double pl_server_now(const pl_server *srv);
pl_status pl_server_load(pl_server *srv, int *queued, int *running,
                         size_t *reserved_bytes, uint64_t *launches);
void pl_server_destroy(pl_server *srv);

/* Truncated law (Section 1's second version of the power law; the cutoffs
 * of Tables 2-6): support k = 1..K,
 *     p(k) = k^-gamma / zeta_K(gamma),  zeta_K(gamma) = sum_{k=1}^{K} k^-gamma,
 * with 0 < gamma <= 64 and 2 <= K <= 1024.  The method is the untruncated
 * one with the finite scaling factor: inverse-CDF draws
 * X = min{k in 1..K : P(X > k) < v} (v = m 2^-53, the same Philox streams),
 * the MLE of Eq. 2 (the root of E_g[ln X] = mean of ln x, searched on the
 * whole real line and bounded to [-64, 64]; a sample of only ones counts one
 * point as 2, as in the untruncated case), and D of Eq. 3 over every
 * t = 1..K.  The form of Eq. 2 is the same in both precision forms; in
 * PL_FP32_BULK the CDF prefix sums and D comparisons are binary32 with
 * compensated accumulation. */
typedef struct {
  double gamma;
  uint64_t K;
  int64_t n;
  int64_t replicates;
  uint64_t cell_id;
} pl_tcell;

/* Draws from the truncated law, nrep rows of n (row r = replicate rep0 + r)
 * at out_dev[r * n]; out_dev: device, uint64[nrep * n].  Errors: PL_EINVAL
 * (gamma outside (0, 64], K outside [2, 1024], n < 1, n > 2^34, nrep < 1,
 * cell_id >= 2^32, rep0 + nrep > 2^32, purpose >= 2^31). */
pl_status pl_sample_truncated(pl_ctx *ctx, double gamma, uint64_t K,
                              uint64_t seed, uint64_t cell_id,
                              uint32_t purpose, uint64_t rep0, int64_t nrep,
                              int64_t n, uint64_t *out_dev, void *stream);

/* Cutoff tables of the truncated law (Tables 2-6): as pl_ks_cutoffs, for
 * pl_tcell cells (1 <= n <= 65535).  gamma_hat_dev_opt: NULL or device
 * double, per-replicate fitted exponents (cells concatenated); D_dev_opt:
 * NULL or device, per-replicate D (double for PL_FP64, float for
 * PL_FP32_BULK).  Fits whose Newton solve hits its cap are counted in
 * newton_capped.  Errors: PL_EINVAL (ncells < 1, nq < 1, q outside (0, 1),
 * a cell outside the ranges above, replicates outside [1, 2^32],
 * cell_id >= 2^32), PL_ENOMEM. */
pl_status pl_ks_cutoffs_truncated(pl_ctx *ctx, const pl_tcell *cells,
                                  int ncells, uint64_t seed, const double *q,
                                  int nq, pl_precision prec, double *cutoffs,
                                  void *D_dev_opt, double *gamma_hat_dev_opt,
                                  void *stream);

/* Fit and D of one data set of the truncated law (values 1..K, int32 on the
 * device, 1 <= n <= 2^31 - 1, 2 <= K <= 1024).  gamma: NaN fits the exponent
 * (Eq. 2 with the finite normaliser; the root on the real line, bounded to
 * [-64, 64]) and evaluates D (Eq. 3, every t = 1..K) there; a value in
 * [-64, 64] evaluates D at that exponent.  gamma_host, D_host: host doubles.
 * Synchronises `stream`.  Errors: PL_EINVAL (arguments, a value outside
 * 1..K). */
pl_status pl_fit_ks_truncated(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                              uint64_t K, double gamma, pl_precision prec,
                              double *gamma_host, double *D_host,
                              void *stream);

/* Bespoke cutoffs (Section 3: the cutoff for the exact N and fitted exponent
 * of the sample, simulated): fit alpha-hat and D of the data set as
 * pl_fit_mle / pl_ks_stat do, simulate R data sets of the same n at
 * alpha-hat (purpose 1, cell_id = request_id; the same simulation as
 * pl_bootstrap_pvalue with B = R), refit each, and return the order
 * statistics D_(floor(R q_j)) of their D for the nq quantiles, and
 * p = #{D_b >= D} / R.  The test rejects at level 1 - q_j when D exceeds
 * cutoff j.  x_dev: device int32[n], values >= xmin.  alpha_hat, D, p: host
 * doubles; cutoffs_host: host double[nq].  Synchronises `stream`.
 * Errors: as pl_bootstrap_pvalue, and q outside (0, 1). */
pl_status pl_bespoke_cutoffs(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                             uint64_t xmin, int64_t R, uint64_t seed,
                             uint64_t request_id, const double *q, int nq,
                             pl_precision prec, double *alpha_hat, double *D,
                             double *p, double *cutoffs_host, void *stream);

/* pl_bespoke_cutoffs for nsets data sets at once: every fit first (one
 * synchronisation), then a single simulation plan holding one cell per data
 * set (alpha-hat_i, xmin_i, n_i, R replicates, cell_id = request_id[i]), so
 * many small requests share the GPU.  Each data set's results equal, bit for
 * bit, those of pl_bespoke_cutoffs on it alone.  x_dev: host array of nsets
 * device pointers (int32 data); n, xmin, request_id: host arrays[nsets].
 * alpha_hat, D, p: host double[nsets]; cutoffs_host: host double[nsets * nq]
 * (row per data set).  Synchronises `stream`.  Errors: as
 * pl_bespoke_cutoffs (the data set at fault named in pl_last_error). */
pl_status pl_bespoke_cutoffs_batch(pl_ctx *ctx, int nsets,
                                   const int32_t *const *x_dev,
                                   const int64_t *n, const uint64_t *xmin,
                                   int64_t R, uint64_t seed,
                                   const uint64_t *request_id, const double *q,
                                   int nq, pl_precision prec, double *alpha_hat,
                                   double *D, double *p, double *cutoffs_host,
                                   void *stream);

/* The same for the truncated law on 1..K (values 1..K, 1 <= n <= 65535):
 * gamma-hat and D as pl_fit_ks_truncated, then R data sets of the same n at
 * (gamma-hat, K) (any gamma-hat in [-64, 64]: the law on a finite support is
 * defined for every real exponent), purpose 1, cell_id = request_id. */
pl_status pl_bespoke_cutoffs_truncated(pl_ctx *ctx, const int32_t *x_dev,
                                       int64_t n, uint64_t K, int64_t R,
                                       uint64_t seed, uint64_t request_id,
                                       const double *q, int nq,
                                       pl_precision prec, double *gamma_hat,
                                       double *D, double *p,
                                       double *cutoffs_host, void *stream);

/* Cutoffs at fitted exponents from a tabulated grid (Section 3: using the
 * tables with a close value of the exponent).  The table holds nq cutoffs
 * for each grid cell (grid_alpha[i], grid_n[k]) at row i * nn + k (the
 * layout pl_ks_cutoffs returns for cells listed exponent-major).  For each
 * query (alpha_dev[m], n_dev[m]) the result is bilinear in (alpha, ln n)
 * between the four surrounding cells, clamped to the grid's edges (so equal
 * to the cell's value at a grid point).  grid_alpha (host, strictly
 * increasing, 1 <= na <= 1024), grid_n (host, strictly increasing, >= 1,
 * 1 <= nn <= 1024);
 * table_dev: device double[na * nn * nq]; alpha_dev, n_dev: device double /
 * int64 [nquery]; out_dev: device double[nquery * nq], row per query.
 * The queries stay on the device and are not checked: an infinite exponent
 * or n = 0 clamps to the grid's edge, a NaN exponent or n < 0 gives NaN.
 * Stream ordered, no synchronisation.  Errors: PL_EINVAL (grids, sizes,
 * null pointers). */
pl_status pl_cutoff_lookup(pl_ctx *ctx, const double *grid_alpha, int na,
                           const int64_t *grid_n, int nn,
                           const double *table_dev, int nq,
                           const double *alpha_dev, const int64_t *n_dev,
                           int64_t nquery, double *out_dev, void *stream);

/* Lower end by KS minimisation (the procedure of Clauset, Shalizi & Newman
 * with which the paper's tables are used, Section 3): every candidate x_min
 * among the smallest max_candidates distinct values of the sample gets the
 * MLE of its tail {x >= x_min} (Eq. 2 with the Hurwitz normaliser; the
 * all-equal rule when the tail is one value) and the tail's D at that fit
 * (Eq. 3); the estimate is the candidate of smallest D (the first on ties).
 * Candidates with fewer than min_tail tail values get D = NaN and are not
 * chosen.  x_dev: device int32[n] (values >= 1, 1 <= n <= 2^31 - 1).
 * out_host: host pl_xmin_result (xmin = 0 and NaN fit if no candidate
 * qualifies).  cand_*_dev: NULL or device arrays of max_candidates entries
 * receiving each candidate's x_min (ascending), alpha-hat, D and tail size
 * (entries beyond `candidates` untouched).  Synchronises `stream`.  The work
 * grows as candidates x distinct values.  Errors: PL_EINVAL (arguments, a
 * value < 1; 1 <= max_candidates <= 2^24, min_tail >= 1). */
typedef struct {
  uint64_t xmin;
  double alpha_hat;
  double D;
  int64_t n_tail;
  int64_t candidates;
} pl_xmin_result;

pl_status pl_estimate_xmin(pl_ctx *ctx, const int32_t *x_dev, int64_t n,
                           int64_t max_candidates, int64_t min_tail,
                           pl_xmin_result *out_host, uint64_t *cand_xmin_dev,
                           double *cand_alpha_dev, double *cand_D_dev,
                           int64_t *cand_ntail_dev, void *stream);

/* Fit and KS distance of one data set with no device allocation at all.
 * The paper has no counterpart: this is an engineering variant of
 * pl_fit_mle + pl_ks_stat for callers that cannot let a library call
 * cudaMalloc -- runtimes that reserve all device memory up front for their
 * own pool allocator, or loops that must never reach the allocator (its
 * calls can synchronise the device).  Its scratch is a fixed device array
 * inside the library (about 6.3 MB on every GPU that loads it, held until
 * the process exits); no context is used.
 * alpha: NaN or <= 0 fits the exponent by maximum likelihood and evaluates D
 *   there; a value in (1, 64] evaluates D at that exponent.
 * x_dev: device int32[n], 1 <= n <= 262144 (larger n: PL_EINVAL), values >= xmin.
 * out_dev: device double[3], written in stream order: alpha (fitted or given),
 *   D, zeta(alpha, xmin); all NaN if a value is below xmin.
 * The first call on each device looks up the array's device address; make
 * that first call before any stream capture.  All calls share the array,
 * which keeps the last call's contents (each call clears what must start at
 * zero); calls that overlap on the GPU race and must be serialised by the
 * caller.  Errors: PL_EINVAL (arguments, n too large), PL_ECUDA. */
pl_status pl_fit_ks_noalloc(const int32_t *x_dev, int64_t n, uint64_t xmin,
                            double alpha, pl_precision prec, double *out_dev,
                            void *stream);

#ifdef __cplusplus
}
#endif

#endif /* PL_H_ */
