/*
 * te_ksg.h -- C ABI of the GB300 (sm_103a) KSG conditional-mutual-information
 * engine and greedy multivariate transfer-entropy network inference.
 *
 * Method: Novelli, Wollstadt, Mediano, Wibral & Lizier, "Large-scale directed
 * network inference with multivariate transfer entropy and hierarchical
 * statistical testing" (Network Neuroscience 2019, arXiv:1902.06828).
 *
 * Conventions used by every entry point
 * -------------------------------------
 * - Every function returns te_status.  On any error the output buffers are left
 *   untouched and te_last_error(ctx) holds a one-line reason until the next call
 *   on that context.  No C++ exception crosses this boundary.
 * - The caller owns every pointer it passes in (inputs and output buffers).
 *   The library owns te_ctx, te_data and te_network_result objects and frees
 *   them through te_ctx_destroy, te_data_destroy and te_network_result_free.
 * - A context is used by one host thread at a time; different contexts are
 *   independent.  All device work of a context runs on its stream (its own
 *   stream by default, or one set with te_ctx_set_stream); blocking calls
 *   synchronise that stream before they return.
 * - Variables are (process, lag) pairs (Methods, "Definitions and assumptions":
 *   the target present Y_t, candidate target past Y_{t-1..t-l_target}, candidate
 *   sources past X_{i,t-1..t-l_sources}).  For an estimate with maximum lag L,
 *   point i (i = 0..N-1, N = T - L) sits at time t_i = L + i, and variable
 *   (p, lag) takes the value series[p][t_i - lag] there.  Lag 0 is the present.
 * - Time series are float32, row-major [n_proc][T], finite values only.
 */
#ifndef TE_KSG_H
#define TE_KSG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TE_OK = 0,
    TE_EINVAL = -1,      /* an argument breaks a documented rule */
    TE_ENOMEM = -2,      /* host or device allocation failed */
    TE_ECUDA = -3,       /* a CUDA runtime call failed (the message names it) */
    TE_ETIMEOUT = -4,    /* te_serve_poll: the job did not finish in time */
    TE_ECANCELLED = -5,  /* te_serve_poll: the job was cancelled */
    TE_EBUSY = -6,       /* te_serve_submit: the job can never fit the device budget */
    TE_EINTERNAL = -7    /* a bug: please report the message */
} te_status;

typedef struct te_ctx te_ctx;
typedef struct te_data te_data;

typedef struct {
    int32_t proc; /* process index, 0 <= proc < n_proc */
    int32_t lag;  /* 0 = present, 1.. = past samples; lag <= the estimate's max lag */
} te_var;

/* Limits of the library. */
#define TE_MAX_DIMS 32      /* dx + dy + dz of one KSG estimate */
#define TE_GAUSS_MAX_DIMS 40 /* dx + dy + dz of one linear-Gaussian estimate (cmi_gauss,
                                te_network_infer with estimator 1) */
#define TE_MAX_K 16         /* nearest neighbours */

/* ---- context and data ---------------------------------------------------- */

/* Create a context on CUDA device `device`.  It owns a stream, a grow-only
 * device workspace and the digamma fixed-point table (see cmi_ksg).
 * Errors: TE_EINVAL (out NULL or bad device), TE_ECUDA, TE_ENOMEM. */
te_status te_ctx_create(int device, te_ctx **out);

/* Run all later work of ctx on `cuda_stream` (a cudaStream_t of the same device,
 * e.g. torch.cuda.current_stream().cuda_stream); NULL restores the context's
 * own stream.  The caller keeps ownership of the stream. */
te_status te_ctx_set_stream(te_ctx *ctx, void *cuda_stream);

void te_ctx_destroy(te_ctx *ctx);

/* One-line reason for the last failed call on ctx ("" after success).  The
 * string stays valid until the next call on ctx.  NULL ctx -> static text. */
const char *te_last_error(const te_ctx *ctx);

/* Copy float32 [n_proc][T] series (host memory when series_on_device == 0,
 * else a device pointer of the context's device) into a device-resident data
 * set owned by the library.  The caller keeps ownership of `series`.
 * Errors: TE_EINVAL (NULL pointers, n_proc < 1, T < 2, a non-finite value),
 * TE_ENOMEM, TE_ECUDA. */
te_status te_data_create(te_ctx *ctx, const float *series, int32_t n_proc, int32_t T,
                         int series_on_device, te_data **out);
void te_data_destroy(te_data *data);

/* Replications (trials) of an experiment (Methods, problem statement: the
 * replication number R; Statistical tests, surrogate paragraph).  `series`
 * is float32 [n_proc][n_rep][T] row-major (host, or device if
 * series_on_device).  Every trial is embedded on its own with the maximum
 * lag L = max_lag and the trials are pooled point by point: the data set
 * holds n_proc * (L + 1) rows of n_rep * (T - L) points, row p * (L + 1) + l
 * being process p at lag l (point r * (T - L) + t = trial r, time L + t - l).
 * te_network_infer takes such data with max(l_target, l_sources) == L and
 * theiler == 0, enumerates candidates over the n_proc processes and draws
 * trial surrogates (te_infer_params.surr_mode).  The single-estimate calls
 * read the rows as processes: variable (p, l) is row p * (L + 1) + l at lag 0,
 * with max_lag 0.
 * Errors: TE_EINVAL (NULL pointers, n_rep < 1, T - max_lag < 2, more than
 * 2^31 pooled values, a non-finite value), TE_ENOMEM, TE_ECUDA. */
te_status te_data_create_trials(te_ctx *ctx, const float *series, int32_t n_proc, int32_t n_rep,
                                int32_t T, int32_t max_lag, int series_on_device, te_data **out);

/* ---- one KSG estimate and its surrogates ---------------------------------- */

typedef struct {
    int32_t k;           /* nearest neighbours, 1..TE_MAX_K (paper: 4) */
    int32_t theiler;     /* Theiler window w >= 0: pairs with |i - j| <= w are
                            excluded from every search (0 = only j == i) */
    int32_t max_lag;     /* L: first point at time L, N = T - L points; every
                            variable's lag must be <= L */
    int32_t n_surr;      /* S >= 0 permutation surrogates of X */
    uint64_t seed;       /* surrogate generator seed */
    uint64_t stream_tag; /* selects an independent surrogate stream */
} te_ksg_params;

/*
 * KSG estimate of the conditional mutual information I(X; Y | Z) and of its
 * S permutation surrogates I(X o pi_s; Y | Z).
 *
 * Estimator (Methods, "Coupled logistic maps process": Kraskov's I^(1) with
 * k nearest neighbours and its extension to CMI; Statistical tests, "Maximum
 * statistic test": surrogates shuffle the embedded source samples, the
 * target is never shuffled):
 *   max-norm distances in float32, d_V(i,j) = max over V's variables of
 *   |v_i - v_j| (the subtraction is the only rounding; d_Z = -inf if dz = 0);
 *   eps_i = k-th smallest max(d_X, d_Y, d_Z) over valid j (j != i, |i-j| > w);
 *   n_xz, n_yz, n_z = numbers of valid j with max(d_X,d_Z), max(d_Y,d_Z), d_Z
 *   strictly below eps_i;
 *   I = psi(k) + (1/N) sum_i [psi(n_z+1) - psi(n_xz+1) - psi(n_yz+1)].
 * The sum is accumulated exactly as the 128-bit integer
 *   K = sum_i (Q[n_z+1] - Q[n_xz+1] - Q[n_yz+1]),  Q[n] = round(2^52 psi(n)),
 * and reported as I = Q[k] 2^-52 + (double)K / (2^52 N), so results do not
 * depend on summation order and every decision is exact.
 *
 * Surrogate s (1..S) reads X at point i from point pi_s(i), pi_s a Fisher-Yates
 * permutation of [0, N) driven by SplitMix64 keyed by (seed, stream_tag, stage
 * 0, iteration 0, s).  Y and Z are never permuted.
 *
 * x, y, z: host arrays of dx >= 1, dy >= 1, dz >= 0 variables (z may be NULL
 * when dz == 0); dx + dy + dz <= TE_MAX_DIMS.
 * out_cmi: host double[1 + S]; [0] is the original estimate, [s] surrogate s.
 * out_key: host int64[2 (1 + S)] or NULL; pairs (hi, lo) of K in two's
 * complement (lo holds the low 64 bits as an unsigned value).
 * Errors: TE_EINVAL (NULL pointers, a variable outside the data, lag > max_lag,
 * max_lag >= T, k outside 1..TE_MAX_K, fewer than k valid neighbours for some
 * point, too many dims, n_surr < 0), TE_ENOMEM, TE_ECUDA.
 */
te_status cmi_ksg(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                  const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                  const te_ksg_params *params, double *out_cmi, int64_t *out_key);

/* Parity/debug form of cmi_ksg for one member (0 = original, s = surrogate s):
 * per-point eps (float[N]) and counts n_xz, n_yz, n_z (int32[N] each) in
 * host memory; any of the four may be NULL.  Same errors as cmi_ksg, plus
 * TE_EINVAL when member is outside 0..n_surr. */
te_status cmi_ksg_debug(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                        const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                        const te_ksg_params *params, int32_t member, float *eps,
                        int32_t *n_xz, int32_t *n_yz, int32_t *n_z);

/* A batch job: one cmi_ksg call (the original plus params.n_surr surrogates). */
typedef struct {
    const te_data *data;
    const te_var *x, *y, *z;
    int32_t dx, dy, dz;
    te_ksg_params params;
} te_cmi_job;

/* Evaluate many jobs in fused launches.  Results are identical to calling
 * cmi_ksg once per job.  out: host double[sum_j (1 + S_j)], jobs in order.
 * out_key: NULL or host int64[2 sum_j (1 + S_j)].  Errors as cmi_ksg (the
 * message names the offending job). */
te_status cmi_ksg_batch(te_ctx *ctx, const te_cmi_job *jobs, int32_t n_jobs, double *out,
                        int64_t *out_key);

/* ---- linear-Gaussian estimate ----------------------------------------------
 *
 * cmi_gauss: the Gaussian (linear) CMI estimate used by the paper for its VAR
 * networks (Methods, Vector autoregressive process; transfer entropy equals
 * Granger causality for Gaussian variables).  The paper prints no formula; the
 * reading used is the plug-in estimate from the sample covariance (ddof = 1) of
 * the embedded variables,
 *   I(X;Y|Z) = 1/2 [ln|S_XZ| + ln|S_YZ| - ln|S_Z| - ln|S_XYZ|]   (|S_Z| = 1 if
 * dz = 0), evaluated as 1/2 [ln|Schur_X given Z| - ln|Schur_X given (Y,Z)|] with
 * FP64 Cholesky factors.  Surrogate s permutes the rows of the whole X block
 * with the same permutation cmi_ksg uses (seed, stream_tag, s); Y and Z are
 * never permuted.  params: max_lag, n_surr, seed, stream_tag are used; k and
 * theiler are ignored.  dx <= 8, dx + dy + dz <= TE_GAUSS_MAX_DIMS (40),
 * N > dx+dy+dz+1.
 * out_cmi: host double[1 + S]; out_err_bound: NULL or host double[1 + S], a
 * first-order bound on |out_cmi - exact FP64 plug-in value| from the error
 * model of the cross-covariance contraction.
 * Errors: TE_EINVAL (as cmi_ksg, dx > 8, too few points, a singular
 * conditioning covariance), TE_ENOMEM, TE_ECUDA. */
te_status cmi_gauss(te_ctx *ctx, const te_data *data, const te_var *x, int32_t dx,
                    const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                    const te_ksg_params *params, double *out_cmi, double *out_err_bound);

/* ---- Theiler-window heuristic ---------------------------------------------- */

/* Autocorrelation decay time (Supporting Information, dynamic correlation
 * exclusion, the heuristic for the Theiler window): the smallest shift
 * tau >= 1 at which the biased sample autocorrelation of process `proc`,
 * r(tau) = sum_{t < T - tau} (x_t - m)(x_{t+tau} - m) / sum_t (x_t - m)^2 with m
 * the series mean, FP64 sums, is <= 1/e (the FP64 number nearest to e^-1);
 * T - 1 if it never is, 1 for a constant series.  proc = -1 gives the largest
 * decay time over all processes.  Blocks until the result is on the host.
 * Errors: TE_EINVAL (proc out of range, T < 2), TE_ENOMEM, TE_ECUDA. */
te_status te_autocorr_decay(te_ctx *ctx, const te_data *data, int32_t proc, int32_t *out_tau);

/* ---- measurement support -------------------------------------------------- */

/* Measured rate of the KSG kernel's counted operations on this GPU, the
 * denominator of that kernel's roofline (measurement support; the paper has no
 * counterpart).  kind 0: the kNN-pass pattern, per member-pair a subtract, a
 * max with d_YZ and one step of the eight-point minimum and threshold compare
 * (3 counted operations); kind 1: the count-pass pattern, per member-pair a
 * subtract, three compares and three predicated increments (7); kind 2: plain
 * FP32 adds (the issue limit, 1 each).  Each probe runs from registers, with
 * the kernel's per-lane shape (4 query points x 2 members x 8-point blocks), at
 * full occupancy for at least 20 ms on the context's stream.  *out_ops_per_s =
 * counted lane operations per second.  Blocks until measured.
 * Errors: TE_EINVAL (kind, NULL), TE_ENOMEM, TE_ECUDA. */
te_status te_alu_peak(te_ctx *ctx, int32_t kind, double *out_ops_per_s);

/* ---- greedy network inference -------------------------------------------- */

typedef struct {
    int32_t k, theiler;            /* estimator parameters, as te_ksg_params; theiler < 0:
                                      automatic, the largest autocorrelation decay time over
                                      the processes (te_autocorr_decay with proc = -1) */
    int32_t max_lag_target;        /* l_target >= 1 */
    int32_t max_lag_sources;       /* l_sources >= 1 */
    int32_t n_surr;                /* S; every test needs S * alpha > 1 */
    double alpha_max, alpha_min, alpha_omnibus, alpha_seq;
    int32_t seq_test;              /* 1: run the step-down stage after the omnibus test */
    int32_t fdr;                   /* 1: Benjamini-Hochberg over targets' omnibus p-values */
    double alpha_fdr;
    uint64_t seed;
    const int32_t *targets;        /* host array of target processes, or NULL = all */
    int32_t n_targets;
    int32_t indep_surr;            /* 0: one permutation per (test, surrogate) shared by the
                                      test's candidates; 1: each candidate c of a test (canonical
                                      order, from 0) draws its own, surrogate s keyed by
                                      s + c * 2^32 (Statistical tests, Maximum statistic test a:
                                      surrogates generated for each candidate) */
    int32_t surr_mode;             /* data from te_data_create_trials only (Statistical tests,
                                      surrogate paragraph): 0 = shuffle the candidate's trial
                                      order when the n_rep! orders cover n_surr, else its samples
                                      inside each trial; 1 = trial order; 2 = inside trials.
                                      Trial order: point r*n + t reads trial sigma(r), sigma a
                                      Fisher-Yates shuffle of the trials; inside trials: one
                                      Fisher-Yates shuffle per trial, trial 0 first, all drawn
                                      from one SplitMix64 stream keyed as the permutations */
    int32_t estimator;             /* 0: KSG (above); 1: the linear-Gaussian estimator of
                                      cmi_gauss (Methods, Vector autoregressive process), k
                                      unused, theiler must be 0, every estimate at most 8 X
                                      and 40 variables in all; decisions then compare the
                                      FP64 estimates, whose cross-covariances are summed in
                                      float-float or FP64 arithmetic (about 1e-13 relative) */
} te_infer_params;

typedef struct {
    int32_t target;
    int32_t n_sel_target;
    te_var *sel_target;            /* selected target past, (proc, lag) ascending */
    int32_t n_sel_sources;
    te_var *sel_sources;           /* selected sources past, ascending */
    double omnibus_cmi, omnibus_p; /* collective TE of the selected sources and its p */
    int32_t omnibus_tested;        /* 1 if the omnibus test ran */
    int32_t significant;           /* 1 if the target keeps sources */
    uint64_t n_estimates;          /* CMI estimates (surrogates included) for this target */
} te_target_result;

typedef struct {
    int32_t n_proc, n_targets;
    te_target_result *targets;
    uint8_t *adjacency;            /* [n_proc * n_proc], adjacency[src * n_proc + tgt] */
    int32_t *min_lag;              /* [n_proc * n_proc], smallest selected lag, 0 = no link */
    uint64_t n_estimates;          /* total CMI estimates */
    double seconds;                /* wall time of the inference */
    int32_t theiler;               /* Theiler window the estimates used */
} te_network_result;

/*
 * Greedy multivariate TE network inference with hierarchical tests (Methods,
 * "Inference algorithm" steps 1-4 and "Statistical tests"), every CMI by the
 * KSG estimator above (or the Gaussian one, params->estimator), every test by S
 * permutation surrogates:
 *   step 1 selects the target past by repeated maximum-statistic tests,
 *   step 2 selects the sources past conditioned on what was selected,
 *   step 3 prunes the sources past with minimum-statistic tests,
 *   step 4 runs the omnibus test on the collective TE;
 *   optional: a step-down test after the omnibus (seq_test) and FDR across
 *   targets (fdr).  A link src -> tgt exists when a variable of src is in the
 *   target's selected sources past.
 * Readings where the paper is silent (all documented with the library):
 * p = #{surrogate statistic > observed} / S, significant iff p < alpha; ties in
 * argmax / argmin go to the first candidate in canonical (proc, lag) order;
 * one permutation per (target, stage, iteration, surrogate) is shared by all
 * candidates of a test; pruning stops at the first significant minimum; a
 * failed omnibus test empties the target's sources.
 * All targets use the same N = T - max(l_target, l_sources) points.
 * Result: library-owned, free with te_network_result_free.
 * Errors: TE_EINVAL (bad parameters, S * alpha <= 1, targets out of range,
 * too few points), TE_ENOMEM, TE_ECUDA.
 */
te_status te_network_infer(te_ctx *ctx, const te_data *data, const te_infer_params *params,
                           te_network_result **out);
void te_network_result_free(te_network_result *res);

/*
 * Request trace of te_network_infer (for verification against an independent
 * implementation of the same greedy loop; Methods, "Inference algorithm" steps
 * 1-4).  With a callback set, every test a target runs is reported once, after
 * its estimates are computed and before its decision is taken:
 *   target, stage (1 target past, 2 sources past, 3 pruning, 4 omnibus,
 *   5 step-down), iteration of the stage (0 for stages 4 and 5),
 *   vars[n_vars]: the candidates in the order of the request (stages 1, 2, 3,
 *   5: one variable per candidate, n_cand == n_vars; stage 4: the selected
 *   sources block, one candidate),
 *   keys[2 * n_cand * (n_surr + 1)]: candidate-major, slot c * (n_surr + 1) + s
 *   (s = 0 the original, s >= 1 surrogate s) as (hi, lo) 128-bit two's
 *   complement pairs: the exact KSG digamma key, or with estimator 1 the
 *   order-preserving integer image of the FP64 estimate.
 * The pointers are valid during the callback only.  Tracing copies every key
 * of a round to the host once per round.  fn = NULL switches tracing off.
 * The callback runs on the calling thread, inside te_network_infer; it must
 * not call into the library with the same context.  Errors: TE_EINVAL for a
 * NULL context.
 */
typedef void (*te_trace_fn)(void *user, int32_t target, int32_t stage, int32_t iter,
                            const te_var *vars, int32_t n_vars, int32_t n_cand,
                            int32_t n_surr, const int64_t *keys);
te_status te_ctx_set_trace(te_ctx *ctx, te_trace_fn fn, void *user);

/* ---- execution options (tuning and measurement; the paper has no counterpart) --
 *
 * te_ctx_set_option sets one option of a context for its later calls:
 *   TE_OPT_KSG_TILE              points per staged tile of the member-lane KSG
 *                                kernel: 64, 128 or 256; 0 (default) = the
 *                                compiled tuning table, chosen by points,
 *                                conditioning dimensions and group size
 *   TE_OPT_KSG_MEMBERS_PER_LANE  1 or 2 (2 only where every group of a launch
 *                                has at least 64 members); 0 (default) = the
 *                                tuning table
 *   TE_OPT_PERSISTENT            1: member-lane launches run as persistent
 *                                grids (as many CTAs as are resident at once,
 *                                each taking query-tile x member-block items
 *                                from a device counter); 0 (default): one CTA
 *                                per item
 *   TE_OPT_GRAPH                 1: each batch's device work (point orders,
 *                                X-value rows, KSG kernels, finalize) is
 *                                captured into a CUDA graph on the context's
 *                                stream and launched as one graph; 0 (default):
 *                                direct launches.  The stream must not be
 *                                capturing already.
 *   TE_OPT_KSG_ORDER             spatial order of the points the KSG kernels
 *                                prune by: 1 = Morton curve, 2 = k-d tree;
 *                                0 (default) = the k-d tree for groups of at
 *                                least 4096 members, the Morton curve below
 * None of them changes a result.  Errors: TE_EINVAL for an unknown option or
 * value. */
#define TE_OPT_KSG_TILE 1
#define TE_OPT_KSG_MEMBERS_PER_LANE 2
#define TE_OPT_PERSISTENT 3
#define TE_OPT_GRAPH 4
#define TE_OPT_KSG_ORDER 5
te_status te_ctx_set_option(te_ctx *ctx, int32_t option, int64_t value);

/* Counters of a context since its creation. */
typedef struct {
    uint64_t estimates;       /* CMI estimates (members) evaluated */
    uint64_t launches;        /* kernel launches issued (all kernels of the library) */
    uint64_t pair_evals;      /* member x point-pair distance evaluations the KSG kernel
                                 executed (both passes; pairs of skipped chunks excluded) */
    double kernel_ms;         /* summed device time of the KSG kernels (CUDA events on the
                                 context's stream) */
    uint64_t ksg_launches;    /* launches of the fused KSG kernel */
    uint64_t h2d_bytes;       /* bytes copied host -> device by the library */
    uint64_t d2h_bytes;       /* bytes copied device -> host by the library */
    uint64_t pair_evals_bruteforce; /* member x ordered point pairs x 2 passes: the work of
                                       the unpruned all-pairs estimator */
    uint64_t ksg_ops;         /* algorithmic ops of the executed evaluations: 3 per kNN-pass
                                 pair (subtract, max, compare), 7 per count-pass pair
                                 (subtract, 3 compares, 3 increments) */
} te_stats;

te_status te_get_stats(const te_ctx *ctx, te_stats *out);

/* ---- serving: continuous batching ------------------------------------------
 *
 * Jobs (te_cmi_job, as for cmi_ksg_batch) are submitted from any host thread
 * and evaluated by a scheduler thread of the context.  Pending jobs are
 * admitted in arrival order while the device memory of the admitted jobs stays
 * within hbm_budget_bytes; each admitted set is fused into one batch, and up to
 * max_inflight batches run on the device at once, each on its own stream.
 * Jobs submitted while batches run join the next batch.  A job's result does
 * not depend on the batch it lands in (exact keys), so it equals cmi_ksg's.
 * Data sets stay resident on the device (te_data) across jobs.
 * (Supporting Information, Run-time on CPU and GPU: targets are independent
 * and may be analysed concurrently.)
 */
typedef uint64_t te_ticket;

typedef struct {
    size_t hbm_budget_bytes;  /* device bytes admitted jobs may hold at once (0: 4 GiB); a job
                                 needs about 12 S N + 4 N (2 + dy + dz) + 64 (S + 1) bytes */
    int32_t max_inflight;     /* batches on the device at once, 1..8 (0: 2) */
    int32_t max_batch_jobs;   /* jobs per batch (0: 2048) */
} te_serve_config;

typedef struct {
    uint64_t submitted, completed, cancelled, batches;
    size_t in_use_bytes, peak_bytes;   /* admitted footprint now / at most */
    uint64_t pending;                  /* jobs waiting for admission */
} te_serve_stats;

/* Start serving on ctx with cfg (NULL: defaults).  te_serve_submit starts it
 * with defaults when needed.  Errors: TE_EINVAL (already started, bad cfg),
 * TE_ECUDA / TE_ENOMEM (streams or host state could not be created). */
te_status te_serve_start(te_ctx *ctx, const te_serve_config *cfg);

/* Queue one job; *out receives its ticket.  The job's arrays are copied, the
 * data set must stay alive until the job is polled.  Thread-safe.
 * Errors: TE_EINVAL (as cmi_ksg), TE_EBUSY (the job alone exceeds the budget). */
te_status te_serve_submit(te_ctx *ctx, const te_cmi_job *job, te_ticket *out);

/* Wait up to timeout_ms (< 0: no limit) for the job, then copy its results:
 * out host double[1 + S], out_key NULL or host int64[2 (1 + S)], as cmi_ksg.
 * A ticket is released by the poll that returns TE_OK, TE_ECANCELLED or an
 * error; TE_ETIMEOUT keeps it.  Thread-safe.  Errors: TE_EINVAL (unknown
 * ticket), TE_ETIMEOUT, TE_ECANCELLED, or the job's CUDA error. */
te_status te_serve_poll(te_ctx *ctx, te_ticket ticket, int32_t timeout_ms, double *out,
                        int64_t *out_key);

/* Cancel a job: a pending job never runs; a running job's results are
 * discarded.  Its next poll returns TE_ECANCELLED.  Thread-safe. */
te_status te_serve_cancel(te_ctx *ctx, te_ticket ticket);

/* Stop serving: pending jobs are cancelled, running batches finish, the
 * scheduler thread exits.  te_ctx_destroy calls it. */
te_status te_serve_stop(te_ctx *ctx);

te_status te_serve_get_stats(te_ctx *ctx, te_serve_stats *out);

/* ---- allocation-free estimate (an addition of this library; the paper has no
 * counterpart) ---------------------------------------------------------------
 *
 * cmi_ksg_static computes exactly what cmi_ksg computes (same estimator, same
 * surrogate permutations, same keys and values) without allocating any device
 * memory, for callers that cannot call cudaMalloc: a host framework that has
 * already reserved the device for its own pool allocator, a serving process
 * that budgets all device memory up front, or a latency-critical loop that
 * cannot afford the device synchronisation of cudaMalloc / cudaFree.
 *
 * Its scratch memory (surrogate permutations, digamma table, launch
 * descriptors, accumulators, keys) is one file-scope device array of
 * TE_STATIC_SCRATCH_BYTES that every GPU which loads this library holds until
 * the process exits.  A call needs the sum of seven parts, each rounded up to
 * a multiple of 256 bytes:
 *   8 (N + 2)            digamma table
 *   4 S N                surrogate permutations
 *   256                  group descriptor (one, at most 256 bytes)
 *   24 (S + 1)           member descriptors
 *   4 (dx + dy + dz)     column offsets
 *   16 (S + 1), twice    key accumulators and keys
 * with N = T - max_lag and S = n_surr <= TE_STATIC_MAX_SURR; it returns
 * TE_EINVAL when the sum exceeds TE_STATIC_SCRATCH_BYTES.
 *
 * series_dev: device float32 [n_proc][T] on the current device, owned by the
 * caller; TE_EINVAL if it is not device memory of the current device.  x, y, z, params: as cmi_ksg.  cuda_stream: a cudaStream_t of the
 * current device or NULL (legacy default stream); the call synchronises it.
 * out_cmi: host double[1 + S]; out_key: NULL or host int64[2 (1 + S)].
 * Errors: status codes only (no context carries a message): TE_EINVAL for any
 * rule cmi_ksg checks plus the scratch limit, TE_ECUDA for a failed CUDA call.
 *
 * The first call on a device resolves the device address of the scratch array
 * (cudaGetSymbolAddress, with that device current).  No call may be made while
 * its stream is being captured into a CUDA graph: each call copies from host
 * staging buffers and synchronises the stream.  All calls share the array,
 * which keeps the last call's contents; each call clears what must start at
 * zero.  Calls whose work overlaps on the GPU race on the array, and calls
 * from several host threads race on static host buffers: serialise them. */
#define TE_STATIC_SCRATCH_BYTES (32u << 20)
#define TE_STATIC_MAX_SURR 4095
te_status cmi_ksg_static(const float *series_dev, int32_t n_proc, int32_t T, const te_var *x,
                         int32_t dx, const te_var *y, int32_t dy, const te_var *z, int32_t dz,
                         const te_ksg_params *params, void *cuda_stream, double *out_cmi,
                         int64_t *out_key);

#ifdef __cplusplus
}
#endif

#endif /* TE_KSG_H */
