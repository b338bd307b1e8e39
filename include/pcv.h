/*
 * pcv.h -- C ABI of the B300 (sm_103a) parallel Bayesian cross-validation
 * library (PCV; "Bayesian cross-validation by parallel Markov chain Monte
 * Carlo", arXiv 2310.07002).
 *
 * One context holds one model, one data set, one CV design and K*L HMC
 * chains (L chains for each of K folds) that advance in lock-step on one
 * GPU (Section 3.3).  The workflow of Section 3 maps to the calls:
 *
 *   Step 1/2  pcv_warmup       full-data chains adapt step size and mass,
 *                              fold chains start from full-data draws and
 *                              run a short discarded warm-up (Section 3.1)
 *   Step 3    pcv_sample       parallel sampling with online accumulators
 *                              (Algorithm A2); callable repeatedly
 *   Step 4    pcv_scores       per-fold elpd and MCSE (eq. cv-score, mc-var)
 *             pcv_diagnostics  per-fold and max R-hat, ESS (Section 4)
 *
 * Conventions shared by every call:
 *   - Every call returns a pcv_status; nothing throws or aborts across the
 *     ABI.  On failure the context keeps a message for pcv_last_error; a
 *     failed pcv_create leaves its message with the calling thread
 *     (pcv_last_error(NULL)).
 *   - "host" pointers are ordinary CPU memory owned by the caller; "device"
 *     pointers are CUDA global memory on the context's device, owned by the
 *     caller.  The library never retains a caller pointer after a call
 *     returns.
 *   - Work is issued on the stream given in pcv_options.cuda_stream (NULL:
 *     the legacy default stream).  Calls that return host results
 *     synchronise that stream before returning; device-result calls are
 *     asynchronous on it.
 *   - Matrices are row-major.
 */
#ifndef PCV_H
#define PCV_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pcv_ctx pcv_ctx;

typedef enum {
    PCV_OK = 0,
    PCV_E_INVALID_ARG = 1,  /* a size, pointer or option is out of range */
    PCV_E_BAD_STATE = 2,    /* call out of order (see the state machine) */
    PCV_E_CUDA = 3,         /* a CUDA runtime error; message has the reason */
    PCV_E_OOM = 4,          /* device allocation failed */
    PCV_E_NUMERIC = 5,      /* non-finite data, or a non-finite state */
    PCV_E_TIMEOUT = 6,      /* a bounded device-side wait ran out */
    PCV_E_UNSUPPORTED = 7   /* valid request this build does not implement */
} pcv_status;

/* Likelihood families (the Appendix B masks apply to all of them). */
typedef enum {
    PCV_GAUSS_LINEAR = 0,   /* y ~ N(x'beta, sigma^2); sigma known or sampled */
    PCV_LOGISTIC = 1,       /* y ~ Bernoulli(sigmoid(x'beta)) */
    PCV_HIER_GAUSS = 2,     /* y ~ N(x'beta + tau z_g(n), sigma^2), z ~ N(0,1) */
    PCV_AR_GAUSS = 3        /* Gaussian on a lagged design, sigma sampled */
} pcv_model_kind;

/* Arithmetic of the leapfrog gradient (the accept test and the online
 * accumulators are FP64 in every mode). */
typedef enum {
    PCV_FP32_SIMT = 0,      /* FP32 CUDA-core kernels */
    PCV_TF32 = 1,           /* tcgen05 tensor cores (kind::tf32), FP32 X and parameter
                               shadows rounded to TF32 in, FP32 accumulate; flat models
                               with p <= 112 */
    PCV_BF16 = 2            /* tcgen05 tensor cores, BF16 X and parameter shadows in,
                               FP32 accumulate; flat models (logistic, Gaussian linear,
                               AR) with p <= 128 */
} pcv_precision;

/*
 * Model.  Parameter vector theta (dimension pcv_dim()):
 *   GAUSS_LINEAR, sigma_known > 0 : beta[p]
 *   GAUSS_LINEAR, sigma_known <= 0: beta[p], log sigma
 *   AR_GAUSS                      : phi[p] (coefficients of the lag columns), log sigma
 *   LOGISTIC                      : beta[p]
 *   HIER_GAUSS                    : beta[p], z[n_groups], log tau, log sigma
 * Priors: beta ~ N(0, beta_prior_sd^2 I); sigma ~ half-N(0, sigma_prior_sd);
 * tau ~ half-N(0, tau_prior_sd); scale parameters are sampled on the log
 * scale with the log-Jacobian added.
 */
typedef struct {
    int32_t kind;              /* pcv_model_kind */
    double beta_prior_sd;      /* > 0 */
    double sigma_known;        /* GAUSS_LINEAR: > 0 known noise sd, <= 0 sampled */
    double sigma_prior_sd;     /* > 0 when sigma is sampled */
    double tau_prior_sd;       /* > 0 (HIER_GAUSS) */
    const int32_t *group;      /* host, N entries in [0, n_groups) (HIER_GAUSS), else NULL */
    int32_t n_groups;          /* HIER_GAUSS only */
    /* host, p flags (1 = covariate in the model), or NULL for all: the
     * covariate-selection mask M_j of Appendix B. An inactive coefficient is
     * held at zero (inverse mass 0), so it leaves the likelihood and the
     * predictive; two contexts that differ only in this mask are the models
     * compared by pcv_compare. */
    const int32_t *active_covariates;
    /* host, p flags, or NULL: a second model, the same one restricted to
     * these covariates (a subset of active_covariates; PCV_E_INVALID_ARG
     * otherwise), whose chains run in the same launches as model A's
     * (Appendix B's parallel evaluation of models by their masks): folds
     * [K, 2K) are model B's copies of folds [0, K) (pcv_num_folds reports
     * 2K), chains [K L, 2 K L) its chains.  B takes A's step size and A's
     * adapted inverse mass restricted to B's covariates, and its chains
     * start from A's full-data draws with B's inactive coefficients at 0.
     * pcv_compare_pair compares the two. first_fold must be 0. */
    const int32_t *active_covariates_b;
} pcv_model;

/* Optional device allocator (the Python binding passes the torch caching
 * allocator).  NULL: cudaMalloc / cudaFree. */
typedef void *(*pcv_alloc_fn)(size_t bytes, void *user);
typedef void (*pcv_free_fn)(void *ptr, void *user);

typedef struct {
    uint64_t seed;             /* Philox4x32-10 key */
    int32_t leapfrog_steps;    /* L_f >= 1 */
    double step_size;          /* > 0 fixed; <= 0 adapted in the full-data warm-up */
    const double *inv_mass_diag; /* host, pcv_dim() entries, or NULL (identity, or adapted
                                    when step_size <= 0) */
    int32_t batch_size;        /* b of eq. bmean, >= 1 (default 50) */
    int32_t hv_buffer;         /* h rows excluded on each side of a test block (default 0) */
    int32_t precision;         /* pcv_precision (default PCV_FP32_SIMT) */
    void *cuda_stream;         /* cudaStream_t, NULL = legacy default stream */
    int32_t store_draws;       /* > 0: also keep up to this many draws per chain of the
                                  held-out log predictive (Algorithm 1 test mode) */
    int32_t acov_max_lag;      /* M for the autocorrelation ESS (default 64, 0 = off) */
    int32_t max_batches;       /* capacity of per-batch summaries (default 1024) */
    int32_t n_fulldata_draws;  /* draws kept per full-data chain as the init pool (default 250) */
    double init_scale;         /* full-data chains start at init_scale * N(0, I) (default 1) */
    int32_t use_graphs;        /* 1: replay iterations as CUDA graphs (default 1) */
    pcv_alloc_fn device_alloc; /* optional allocator (see above) */
    pcv_free_fn device_free;
    void *alloc_user;
    /* Trajectory length and step-size jitter. The paper reuses the full-data
     * step size and trajectory length for every fold (Section 3.1); with
     * leapfrog_steps fixed, an adapted step size is capped at
     * trajectory_length / leapfrog_steps (trajectory_length in units of the
     * adapted inverse mass; < 0: pi/2 when the step size is adapted, 0: no
     * cap). Fold chains then draw one step size per iteration, shared by all
     * chains, eps (1 + step_jitter (2u - 1)) with u from Philox stream 3,
     * which breaks the periodicity of a fixed trajectory (Neal 2011).
     * step_jitter < 0: 0.5 when the step size is adapted, else 0; must be
     * < 1. */
    double trajectory_length;
    double step_jitter;
    /* 1 (default): before the first iterations of a chain set, time the
     * gradient launch under a few launch configurations (split-N count of
     * the FP32 kernels, X pipeline depth of the tensor-core kernel) and keep
     * the fastest for that chain count. The split count changes the order of
     * the FP32 partial sums, so results are bit-reproducible only with the
     * same choice; 0 keeps the fixed rule. */
    int32_t autotune;
    /* bit 0: accumulate the Hyvarinen score (Algorithm A3), bit 1: the
     * Dawid-Sebastiani score (Algorithm A4), read with pcv_scores_extra.
     * Gaussian linear and AR models only (rows conditionally independent
     * given theta); the DSS needs test sets of at most 64 rows. Default 0. */
    int32_t extra_scores;
    /* Global id of this context's fold 0 when the folds of one problem are
     * split over several contexts (one per GPU): the Philox counters of fold
     * chain c use chain id first_fold * L + c and the shuffle benchmark fold
     * id first_fold + k, so every fold draws the same random numbers however
     * the folds are split. Default 0. */
    int32_t first_fold;
    /* Whole leapfrog trajectories in one launch for small problems (flat
     * models, p <= 32, FP32 or BF16 form; Section 3.3's lock-step HMC needs
     * no synchronisation between chains, so a team of 1, 2, 4 or 8 warps
     * carries one chain through the momentum draw and all L_f gradient
     * steps, its rows split over the team): -1 (default) lets the autotuner
     * time it, with each team size, against k_begin + L_f gradient launches
     * per chain count (without the autotuner: rows x register width <= 32 Ki
     * takes it, with teams that fill the GPU); 0 never; 1, 2, 4 or 8: always
     * where the problem allows it, with that many warps per chain. */
    int32_t fused_trajectory;
    /* Tensor-core forms (BF16, TF32), where each 128-chain tile has a CTA of its own
     * (the autotuner's grid for short tiles, e.g. leave-one-out on a few
     * thousand rows): 0 (default) runs the L_f - 1 kick-drift steps of a
     * trajectory in one launch, each CTA carrying its tile from step to step
     * (lock-step HMC, Section 3.3: a tile depends on no other tile); 1 runs
     * one launch per step. Both give the same bits. */
    int32_t tc_steps_per_launch;
    /* Tensor-core grid: 0 (default) the autotuner's choice per chain count;
     * 1 one CTA per SM with the chain tiles split across CTAs (stream-K);
     * 2 one CTA per 128-chain tile. Fixing it makes profiler runs (where
     * the autotuner's timings are distorted) take the grid of a live run. */
    int32_t tc_grid;
} pcv_options;

/* Fill *opt with the defaults listed above (seed 0, L_f 16, adapted step). */
void pcv_default_options(pcv_options *opt);

/*
 * Create a context (state: created).
 *   X               host, N x p row-major, finite
 *   y               host, N, finite (LOGISTIC: 0 or 1)
 *   fold_assignment host, N; fold of each row in [0, K) or -1 for rows that are
 *                   in no test set; every fold 0..K-1 must appear.  With
 *                   hv_buffer > 0 each fold's test rows must be contiguous.
 *   chains_per_fold L >= 2 (R-hat needs two chains)
 * Rows are re-ordered internally so that each fold's test rows (and, for
 * HIER_GAUSS, each group) are contiguous; results do not depend on the
 * caller's row order except through hv_buffer.  X, y and the fold layout are
 * copied to device memory owned by the context.  The fold masks are those
 * of eq. mask-log-prob / mask-log-pred (Appendix B), the training mask being
 * the complement of the test mask (minus the h(v)-block buffer).
 * Errors: INVALID_ARG (N < 1, p < 1, L < 2, a fold with no test or no
 * training rows, missing fold ids, bad option), NUMERIC (non-finite data),
 * UNSUPPORTED (precision/model/size combination not built), OOM, CUDA.
 */
pcv_status pcv_create(const pcv_model *model, const float *X, const float *y,
                      const int32_t *fold_assignment, int64_t N, int32_t p,
                      int32_t chains_per_fold, const pcv_options *opt, pcv_ctx **out);

/*
 * Warm-up reuse (Section 3.1; Algorithm 1 before its sampling loop):
 * 4 full-data chains run n_fulldata_warmup adaptation iterations (dual
 * averaging of the step size toward acceptance 0.8 unless a step size was
 * given; a diagonal inverse mass from iterations [n/4, n/2) unless one was
 * given) and n_fulldata_draws kept iterations; each fold chain starts from a
 * full-data draw chosen uniformly with replacement and runs n_fold_warmup
 * discarded iterations.  State: created -> warmed.  May be called once.
 */
pcv_status pcv_warmup(pcv_ctx *ctx, int32_t n_fulldata_warmup, int32_t n_fold_warmup);

/*
 * Draw n_draws (a positive multiple of batch_size) HMC iterations for all
 * K*L chains and feed each draw of s = log p(y_test_k | theta) into the
 * online accumulators (Algorithm A2).  Repeatable: later calls continue the
 * same chains and accumulators (progressive estimates).  State: warmed or
 * sampled -> sampled.
 */
pcv_status pcv_sample(pcv_ctx *ctx, int32_t n_draws);

/*
 * Scores (host outputs, caller-owned; any pointer may be NULL):
 *   elpd_k[K]   log of the Monte Carlo mean of p(y_test_k | theta)  (eq. cv-score term)
 *   mcse_k[K]   its MCSE by batch means and the delta method     (eq. bmvar, mc-var)
 *   elpd_total  sum of elpd_k; mcse_total = sqrt(sum mcse_k^2)
 *   se_epistemic sqrt(K var_k(elpd_k))                          (eq. norm-approx)
 * Needs at least 2 batches sampled (BAD_STATE otherwise).
 */
pcv_status pcv_scores(pcv_ctx *ctx, double *elpd_k, double *mcse_k, double *elpd_total,
                      double *mcse_total, double *se_epistemic);

/*
 * Diagnostics on the s draws (host outputs, caller-owned; any may be NULL):
 *   rhat_k[K]        eq. rhat (no splitting, no rank normalisation)
 *   split_rhat_k[K]  eq. rhat over 2L half chains made of whole batches
 *   ess_bm_k[K]      L n s^2 / sigma^2_bm of exp(s)              (Section 4.1)
 *   ess_acov_k[K]    multi-chain autocorrelation ESS of s (Geyer initial
 *                    monotone sequence, lags <= acov_max_lag)
 *   divergences_k[K] divergent transitions while sampling
 *   rhat_max         max_k rhat_k                                (eq. rhat-max)
 *   ess_total        aggregate ESS over folds                    (Section 4.1)
 */
pcv_status pcv_diagnostics(pcv_ctx *ctx, double *rhat_k, double *split_rhat_k,
                           double *ess_bm_k, double *ess_acov_k, int64_t *divergences_k,
                           double *rhat_max, double *ess_total);

int32_t pcv_num_folds(const pcv_ctx *ctx);    /* K, or -1 for NULL */
int32_t pcv_num_chains(const pcv_ctx *ctx);   /* K * L */
int32_t pcv_dim(const pcv_ctx *ctx);          /* dimension of theta */
/* Never NULL; valid until the next call. With ctx == NULL: the message of
 * the calling thread's last failed pcv_create ("null context" if none). */
const char *pcv_last_error(const pcv_ctx *ctx);
void pcv_destroy(pcv_ctx *ctx);               /* frees all device memory; NULL is a no-op */

/* ---------------- inspection and test entry points ---------------- */

/*
 * Set every fold chain's position (host, C x dim, chain c = k*L + l) and,
 * optionally, the step size (> 0) and inverse mass (host, dim; NULL keeps
 * it), instead of pcv_warmup.  Recomputes log densities and gradients.
 * State: created/warmed -> warmed (accumulators untouched).
 */
pcv_status pcv_set_positions(pcv_ctx *ctx, const double *theta, double step_size,
                             const double *inv_mass_diag);

/* Current positions (host C x dim), log posterior and held-out log
 * predictive at them (host C each); any pointer may be NULL. */
pcv_status pcv_get_positions(pcv_ctx *ctx, double *theta, double *logp, double *shat);

/* Step size and inverse mass (host, dim) in use. */
pcv_status pcv_get_adaptation(pcv_ctx *ctx, double *step_size, double *inv_mass_diag);

/*
 * Evaluate, for n (position, fold) pairs, the fold-masked log posterior
 * (eq. mask-log-prob + log prior), its gradient and the held-out log
 * predictive (eq. mask-log-pred) with the kernels of the given precision.
 *   theta   device, n x dim FP32
 *   fold    device, n fold ids in [0, K]; K means the full data set
 *   logp    device, n FP64 (out)      grad device, n x dim FP32 (out)
 *   shat    device, n FP64 (out)
 * Uses the context's workspace.  Asynchronous on the context stream.
 */
pcv_status pcv_log_density(pcv_ctx *ctx, const float *theta, const int32_t *fold, int32_t n,
                           int32_t precision, double *logp, float *grad, double *shat);

/*
 * One leapfrog trajectory (L_f steps, Section 3.3) for every fold chain from
 * the given start: theta0, r0 device C x dim FP32.  Outputs (device):
 * theta1, r1 C x dim FP32; logp1, shat1 C FP64.  Uses the context's step
 * size and inverse mass.  Does not change the chains.
 */
pcv_status pcv_trajectory(pcv_ctx *ctx, const float *theta0, const float *r0, int32_t precision,
                          float *theta1, float *r1, double *logp1, double *shat1);

/*
 * Standard normals the sampler draws for (iteration, stream): device out,
 * C x dim FP32, chain c in row c.  Streams: 0 fold momentum, 16 full data.
 */
pcv_status pcv_draw_normals(pcv_ctx *ctx, uint32_t iteration, uint32_t stream, float *out);

/*
 * Feed n given draws per chain (device, C x n FP64) to the online
 * accumulators, as if sampled.  n must be a multiple of batch_size.
 * State: warmed/sampled -> sampled.
 */
pcv_status pcv_accumulate(pcv_ctx *ctx, const double *shat, int32_t n);

/* Stored draws (host, C x n_stored FP64) when store_draws > 0; *n_stored out. */
pcv_status pcv_get_draws(pcv_ctx *ctx, double *shat, int32_t *n_stored);

/* Mean acceptance rate per fold over sampling (host, K). */
pcv_status pcv_accept_rate(pcv_ctx *ctx, double *accept_k);

/*
 * Hyvarinen and Dawid-Sebastiani scores per fold and in total (positively
 * oriented), from the accumulators enabled by pcv_options.extra_scores:
 *   HS_k  = sum_i [-2 E(d2 log p/dy_i^2 + (d log p/dy_i)^2) + (E d log p/dy_i)^2]
 *           over the fold's test rows i, expectations over every fold-chain
 *           draw (Algorithm A3, per test observation);
 *   DSS_k = -log|S_k| - (y - m_k)' S_k^{-1} (y - m_k), m_k and S_k the mean and
 *           covariance of one predictive draw per chain and iteration
 *           (Algorithm A4; draws from Philox stream 5).
 * Host outputs: hs_k, dss_k (K each, or NULL for a score not enabled),
 * hs_total, dss_total. PCV_E_UNSUPPORTED if neither score was enabled,
 * PCV_E_BAD_STATE before pcv_sample.
 */
pcv_status pcv_scores_extra(pcv_ctx *ctx, double *hs_k, double *dss_k, double *hs_total, double *dss_total);

/*
 * Pairwise model selection (eq. sel-cv, eq. norm-approx, eq. mc-var) between
 * model A (ctx_a) and model B (ctx_b), two contexts sampled on the same data
 * and folds (typically the same model with different covariate masks):
 *   delta_k = elpd_A,k - elpd_B,k (host, K), mcse_k = sqrt(MCSE_A,k^2 +
 *   MCSE_B,k^2) (host, K), and out[4] = {delta = sum_k delta_k,
 *   se = sqrt(K var_k(delta_k)), MCSE of delta = sqrt(sum_k mcse_k^2),
 *   Pr(A better than B) = Phi(delta / se)}.
 * Both contexts need pcv_sample first (PCV_E_BAD_STATE); different N or K
 * give PCV_E_INVALID_ARG.
 */
pcv_status pcv_compare(pcv_ctx *ctx_a, pcv_ctx *ctx_b, double *delta_k, double *mcse_k, double *out);

/*
 * The same comparison within one context that runs two models
 * (pcv_model.active_covariates_b): model A's folds [0, K) against model B's
 * [K, 2K); outputs as pcv_compare (delta_k, mcse_k: host, K each; out[4]).
 * PCV_E_INVALID_ARG for a one-model context, PCV_E_BAD_STATE before
 * pcv_sample.
 */
pcv_status pcv_compare_pair(pcv_ctx *ctx, double *delta_k, double *mcse_k, double *out);

/*
 * Kernels the library's iterations (warm-up and sampling) have issued since
 * pcv_create: each iteration graph's kernel nodes, counted at capture, times
 * its replays (no paper counterpart; for benchmark records).  *n out.
 * PCV_E_UNSUPPORTED when iterations ran outside CUDA graphs (use_graphs 0).
 */
pcv_status pcv_kernel_launches(pcv_ctx *ctx, int64_t *n);

/*
 * R-hat_max benchmark (Section 4.2; the block-shuffle loop of Algorithm A2):
 * each chain's draws so far are cut into n_blocks contiguous blocks of whole
 * batches (block d holds batches [d a / D, (d+1) a / D), a batches); each of
 * n_reps replicates rebuilds every chain of every fold from blocks of that
 * fold's chains drawn uniformly with replacement (Philox stream 4; pick
 * t = l D + d of replicate r in fold k is word t % 4 of counter
 * (t / 4, k, r, 4), chain floor(w L / 2^32)) and takes the R-hat (eq. rhat)
 * of the rebuilt chains. rhat_max_rep (host, n_reps) receives the maximum
 * over folds of each replicate: the histogram against which R-hat_max is
 * read; rhat_fold_rep (host, n_reps x K, or NULL) the per-fold values.
 * Needs pcv_sample first (PCV_E_BAD_STATE) and n_blocks <= batches <=
 * max_batches (PCV_E_INVALID_ARG).
 */
pcv_status pcv_rhat_shuffle(pcv_ctx *ctx, int32_t n_blocks, int32_t n_reps, double *rhat_max_rep,
                            double *rhat_fold_rep);

/*
 * Checkpoint / resume (progressive reporting, Section 1: a run can be
 * stopped, reported and continued). A checkpoint holds everything the next
 * iterations read: iteration counters and adaptation state, step size and
 * inverse mass, fold-chain positions, gradients and log densities, the
 * centring reference (tensor-core path), every online accumulator, stored
 * draws, and the autotuner's choices, behind a header that identifies the
 * problem and the options. Loading it into a context created with the same
 * model, data and options (and no warm-up) continues the run bit for bit.
 *   pcv_checkpoint_size: *bytes = the buffer size the save needs.
 *   pcv_checkpoint_save: host buffer buf (caller-owned, >= that size);
 *     PCV_E_BAD_STATE before warm-up or pcv_set_positions.
 *   pcv_checkpoint_load: PCV_E_INVALID_ARG if the buffer is not a
 *     checkpoint, is truncated, or belongs to another problem or options.
 */
pcv_status pcv_checkpoint_size(pcv_ctx *ctx, int64_t *bytes);
pcv_status pcv_checkpoint_save(pcv_ctx *ctx, void *buf, int64_t bytes);
pcv_status pcv_checkpoint_load(pcv_ctx *ctx, const void *buf, int64_t bytes);

/* The launch configurations the autotuner chose (pcv_options.autotune), one
 * line per chain set: the candidates with their measured time per launch
 * and the choice. Writes a NUL-terminated string of at most len bytes
 * (truncated if longer) into buf, a host buffer the caller owns. No
 * counterpart in the paper. */
pcv_status pcv_tuning_info(const pcv_ctx *ctx, char *buf, int32_t len);

/* Host wall-clock milliseconds that the context has spent, so far, in the
 * autotuner (*autotune_ms: timing candidate launch configurations, once per
 * chain set) and in capturing and instantiating CUDA graphs
 * (*graph_capture_ms: once per kind of iteration). Both are part of the
 * pcv_warmup / pcv_sample wall clock; they are reported apart because they
 * do not recur. Host pointers, caller-owned; PCV_E_INVALID_ARG if any is
 * null. No counterpart in the paper. */
pcv_status pcv_setup_ms(const pcv_ctx *ctx, double *autotune_ms, double *graph_capture_ms);

/* Device time in milliseconds of the most recent pcv_sample call (CUDA events
 * on the context stream). */
pcv_status pcv_last_sample_ms(pcv_ctx *ctx, double *ms);

/*
 * Time the fused leapfrog gradient kernel exactly as sampling launches it
 * (one kick-drift step for all fold chains, Section 3.3): `reps` launches on
 * the context stream between two CUDA events; *ms_per_launch receives the
 * mean.  Only the proposal buffers change (the next iteration overwrites
 * them); needs warmed positions.
 */
pcv_status pcv_time_leapfrog_kernel(pcv_ctx *ctx, int32_t reps, double *ms_per_launch);

/*
 * The pool of full-data draws that fold chains start from (Algorithm 1,
 * "draw from {theta^(fd)}"; warm-up reuse, Section 3.1), after pcv_warmup:
 * *n_pool = 4 x n_fulldata_draws rows; when pool is not NULL it receives
 * them as [n_pool x dim] doubles (row i x 4 + c = full-data chain c after
 * kept iteration i), in caller-owned host memory.  Fold chain c starts from
 * row floor(w0 n_pool / 2^32), w0 the first Philox word of (block 0, chain
 * first_fold x L + c, iteration 0, stream 2).  PCV_E_BAD_STATE before the
 * warm-up.
 */
pcv_status pcv_get_pool(pcv_ctx *ctx, double *pool, int32_t *n_pool);

/*
 * Test entry for the full-data adaptation arithmetic (warm-up reuse,
 * Section 3.1: dual averaging of the step size, Hoffman & Gelman 2014, and
 * the two diagonal-mass windows [n/4, n/2) and [n/2, 7n/8)): runs the
 * adaptation kernel n_adapt times on given inputs instead of HMC
 * transitions.  accept [n_adapt x 4] holds the acceptance statistic of each
 * of the 4 full-data chains after iteration i, draws [n_adapt x 4 x dim]
 * (FP32) their positions; the step size starts at eps0 > 0 and the inverse
 * mass at the context's.  Outputs (caller-owned host memory): eps_out
 * [n_adapt] and minv_out [n_adapt x dim], the step size and inverse mass
 * after each iteration, and *eps_final, the dual-averaged step size with no
 * cap.  Only before pcv_warmup (PCV_E_BAD_STATE otherwise); the context's
 * inverse mass is restored afterwards and pcv_warmup starts afresh.
 */
pcv_status pcv_adapt_trace(pcv_ctx *ctx, int32_t n_adapt, const double *accept, const float *draws,
                           double eps0, int32_t adapt_mass, double *eps_out, double *minv_out,
                           double *eps_final);

/*
 * Allocation-free gradient evaluation (the paper has no counterpart).  It is
 * for callers that may not allocate device memory while they run: a process
 * whose GPU memory belongs to another framework's pool, or a latency-bound
 * loop where cudaMalloc could block or synchronise the device.  The kernels'
 * split-N partial sums and tickets live in fixed device arrays compiled into
 * the library (16 MiB of FP32 scratch and 8192 tickets; every GPU that loads
 * the library holds them until the process exits) instead of the context's
 * workspace, so the call itself allocates nothing.
 *   - Arguments, layout and results as pcv_log_density, except the
 *     precision: it must be PCV_FP32_SIMT, and the call runs the FP32
 *     CUDA-core gradient kernel on a context of any precision (the context
 *     keeps the FP32 design matrix on every path), so on a BF16 or TF32
 *     context it returns FP32 results where pcv_log_density would return the
 *     context's precision.
 *   - Limits, with T chains per tile (T = 32 for p <= 32, T = 64 above) and
 *     W = max(dim rounded up to 4, the kernel's register width for p <= 32)
 *     + 4 partial sums per chain: ceil(n / T) <= 8192 tiles (one ticket each)
 *     and ceil(n / T) * T * W <= 4 Mi floats for one split of the rows; the
 *     split count is the one pcv_log_density would use, reduced if needed so
 *     that all splits fit.  Larger n returns PCV_E_INVALID_ARG with a message
 *     naming the limit.
 *   - The first call on a device looks up the arrays' device addresses
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 *   - All calls share the arrays, which keep the previous call's contents
 *     (the tickets are cleared at the start of each call): calls that can
 *     overlap on the GPU, from any context or stream, race and must be
 *     serialised by the caller.
 */
pcv_status pcv_log_density_noalloc(pcv_ctx *ctx, const float *theta, const int32_t *fold,
                                   int32_t n, int32_t precision, double *logp, float *grad,
                                   double *shat);

#ifdef __cplusplus
}
#endif
#endif /* PCV_H */
