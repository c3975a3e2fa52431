/*
 * smc.h -- C ABI of the B300 (sm_103a) SMC hot path.
 *
 * The calls follow the decomposition of a vSMC sampler (Zhou, "vSMC:
 * Parallel Sequential Monte Carlo in C++", arXiv 1306.5583):
 *   Sampler(N, scheme, threshold)          -> smc_config, smc_create
 *   Sampler::initialize                    -> smc_initialize
 *   one iteration = move queue, ESS test and resampling, mcmc queue,
 *   monitors (Sec. 4.1.3)                  -> smc_move, smc_resample, smc_mcmc
 *   Sampler::iterate(n)                    -> smc_iterate
 *   (there is no separate smc_weight or smc_run: the weight update,
 *   normaliser and ESS test of a particle filter are part of smc_move --
 *   vSMC's move queue -- and a run of iterations is smc_iterate; for the GMM
 *   sampler smc_move is the reweighting at alpha_t and smc_mcmc the
 *   Metropolis / Langevin moves)
 *   WeightSet::add_log_weight (Sec. 4.1.6) -> smc_add_log_weight
 *   NormalizingConstant / Path estimates   -> smc_log_evidence, smc_path_sampling
 *   read_weight / read_log_weight          -> smc_read_log_weight
 *   copy(N, copy_from) convention (Sec. 4.1.2): ancestors[k] is the parent
 *   of new particle k                      -> smc_read_ancestors
 *
 * Conventions shared by every call
 * * Return value: SMC_OK (0) or one of the SMC_E_* codes below.  No C++
 *   exception crosses this boundary.
 * * Device work is queued on the CUDA stream given to smc_create and runs
 *   asynchronously; errors raised on the device (non-finite weights, a
 *   bounded wait that gave up) are kept in a device error word and returned
 *   by the next call that synchronises (smc_ess with a host pointer,
 *   smc_log_evidence, smc_path_sampling, smc_read_*, smc_sync).  smc_read_*
 *   still copy their data when the error word is set (the particle system of
 *   a failed step is the one before it) and return the error.
 * * Memory: the caller owns the device workspace (size from
 *   smc_workspace_bytes, 256-byte aligned) and the stream; the context holds
 *   non-owning pointers into them and host memory of its own.  Host buffers
 *   passed to smc_read_* are caller-owned.  `on_device` arguments say
 *   whether a pointer is device memory (1) or host memory (0).
 * * Threading: one context must not be used by two threads at once;
 *   distinct contexts are independent (the thread-safety rules of Sec. 4.3).
 * * Random numbers: Philox4x32-10 (Salmon et al., SC'11; the paper's
 *   per-particle counter-based streams, Sec. 3.4) with key = (seed low 32
 *   bits, seed high 32 bits) and counter = (particle or slot index,
 *   iteration t, purpose tag | stream_id << 16, draw index).
 */
#ifndef SMC_H
#define SMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SMC_OK 0
#define SMC_E_ARG 1        /* invalid argument or configuration */
#define SMC_E_WORKSPACE 2  /* workspace too small or misaligned */
#define SMC_E_NONFINITE 3  /* all weights zero or NaN: state left untouched */
#define SMC_E_TIMEOUT 4    /* a bounded device wait gave up */
#define SMC_E_CUDA 5       /* a CUDA runtime call failed */
#define SMC_E_STATE 6      /* call out of order (e.g. move before initialize) */
#define SMC_E_RANGE 7      /* a device counter left its range: a 24-bit multinomial or
                            * residual draw value drawn 256 times in one resampling step
                            * (probability below 1e-60 per step for N <= 2^30); the
                            * step's ancestors are not valid */

/* resampling schemes (Sec. 2.1; Douc et al. 2005); the paper's default is
 * stratified (Sec. 4.1.3) */
#define SMC_MULTINOMIAL 0
#define SMC_STRATIFIED 1
#define SMC_SYSTEMATIC 2
#define SMC_RESIDUAL 3              /* floor(N W_i) copies, then multinomial on the residual weights */
#define SMC_RESIDUAL_SYSTEMATIC 4   /* the same copies, the R residual outputs drawn systematically */
#define SMC_RESIDUAL_STRATIFIED 5   /* ... or stratified (Douc et al. 2005 list both variants) */

/* config flags */
#define SMC_FLAG_KEEP_CDF 1u  /* store the fixed-point CDF of each resampling step (smc_read_cdf) */
#define SMC_FLAG_RECORD 2u    /* CV models: record the ancestors of every step and a state checkpoint
                                 every checkpoint_every steps, for smc_pf_grad / smc_pf_replay */
#define SMC_FLAG_POST_MEAN 4u /* CV models: also record the post-resampling filtered mean (mean_post;
                                 Sec. 4.1.5 evaluates monitors after the whole iteration) with one
                                 more kernel after each resampling step */
#define SMC_FLAG_INPLACE 8u   /* arrange each step's ancestors in place (copy_from of Sec. 4.1.2):
                                 a particle with offspring keeps its own slot, the extra copies fill
                                 the slots of particles without offspring in increasing order
                                 (smc_read_ancestors then returns that arrangement); one more kernel
                                 after each resampling step; not with SMC_FLAG_RECORD */

/* models */
#define SMC_MODEL_CV 0        /* Sec. 5.1: constant-velocity tracking, Student-t observations */
#define SMC_MODEL_CV_GAUSS 1  /* same with Gaussian observations (Kalman closed form) */
#define SMC_MODEL_GMM 2       /* Sec. 5.2: Bayesian Gaussian mixture, tempered SMC sampler */

/* GMM mcmc moves: the paper's three random-walk Metropolis blocks, a
 * Metropolis-adjusted Langevin move on all unconstrained coordinates driven by
 * the gradient of the tempered log-target, or the blocks followed by one
 * Langevin move */
#define SMC_GMM_RW 0
#define SMC_GMM_MALA 1
#define SMC_GMM_RW_MALA 2

/* GMM annealing schedules (Sec. 5.2.3) */
#define SMC_ALPHA_LINEAR 0  /* alpha_t = t / T */
#define SMC_ALPHA_PRIOR 1   /* alpha_t = (t / T)^p */
#define SMC_ALPHA_ADAPTIVE 2 /* alpha_t chosen on the device at every iteration so that the conditional
                                ESS of the incremental weights, N (sum W_i w_i)^2 / sum W_i w_i^2 with
                                w_i = exp((alpha_t - alpha_{t-1}) l_i), equals ess_target N (or
                                alpha_t = 1 when it stays above that at alpha = 1): 40 halvings of
                                [0, 1 - alpha_{t-1}] in one cooperative kernel; the chosen alpha_t
                                is in the record; later iterations keep alpha = 1 */

/* Almost-constant-velocity model parameters (Sec. 5.1.1). */
typedef struct {
    double delta;      /* time step Delta */
    double sd_pos;     /* process-noise sd on positions */
    double sd_vel;     /* process-noise sd on velocities */
    double obs_scale;  /* observation-noise scale s */
    double obs_df;     /* Student-t degrees of freedom nu */
    double sd_pos0;    /* prior sd of the positions at t = 0 */
    double sd_vel0;    /* prior sd of the velocities at t = 0 */
} smc_cv_params;

/* Gaussian-mixture model and sampler parameters (Sec. 5.2.1-5.2.3). */
typedef struct {
    int32_t n_comp;       /* r, 1..8 */
    int32_t schedule;     /* SMC_ALPHA_LINEAR, SMC_ALPHA_PRIOR or SMC_ALPHA_ADAPTIVE */
    int32_t n_iter;       /* T_r: alpha reaches 1 at t = T_r (adaptive: the most iterations) */
    int32_t shape0;       /* Gamma prior shape of each precision (integer >= 1) */
    double power;         /* p of the prior schedule */
    double mu0, sd0;      /* normal prior of each mean */
    double rate0;         /* Gamma prior rate of each precision */
    int32_t move;         /* SMC_GMM_RW, SMC_GMM_MALA or SMC_GMM_RW_MALA */
    int32_t reserved;
    double mala_step;     /* Langevin step size epsilon */
    double ess_target;    /* SMC_ALPHA_ADAPTIVE: rho in (0, 1), the conditional ESS target rho N */
} smc_gmm_params;

typedef struct {
    int32_t model;        /* SMC_MODEL_* */
    int32_t precision;    /* 32: FP32 per particle, FP64 normaliser and evidence;
                             64: FP64 throughout */
    int64_t n_particles;  /* 1 <= N <= 2^30 (smc_create refuses others) */
    int32_t max_records;  /* iteration records kept on the device (ring), >= 2 */
    int32_t scheme;       /* SMC_* resampling scheme */
    double threshold;     /* resample when ESS < threshold * N; >= 1 always, <= 0 never */
    uint64_t seed;        /* Philox key */
    uint32_t stream_id;   /* Philox stream (counter word 2, high 16 bits) */
    uint32_t flags;       /* SMC_FLAG_* */
    int64_t max_data;     /* capacity for observations: CV rows (Y_0..), GMM points */
    smc_cv_params cv;
    smc_gmm_params gmm;
    int32_t checkpoint_every; /* SMC_FLAG_RECORD: steps between state checkpoints (0: 16) */
    int32_t reserved2;
} smc_config;

/* One record per iteration, kept on the device (ring of max_records). */
typedef struct {
    double log_norm;      /* L_t: log-sum-exp of lw_t = log of the estimated Z_t / Z_{t-1} */
    double log_evidence;  /* running sum of L_t (standard estimate, Sec. 2.2) */
    double ess;           /* 1 / sum W_t^2 (Sec. 2.1) */
    double mean[2];       /* PF: filtered means of the positions (before resampling) */
    double max_lw;        /* max_i lw_t,i */
    double path_u;        /* GMM: U_t (eq:path_import) */
    double path_log_z;    /* GMM: running path-sampling estimate (eq:path_est) */
    double alpha;         /* GMM: alpha_t */
    double accept[3];     /* GMM: acceptance rate of the mu, lambda, weight blocks */
    int32_t t;            /* iteration index */
    int32_t resampled;    /* 1 when the ESS test asked for resampling */
    int32_t status;       /* SMC_OK or an error code */
    int32_t pad;
    double accept_mala;   /* GMM: acceptance rate of the Langevin move */
    double mean_post[2];  /* PF with SMC_FLAG_POST_MEAN: mean of the positions over the particle system
                             that ends the iteration (1/N sum_k pos_{a_k} after resampling, else the
                             weighted mean); NaN without the flag */
} smc_record;

typedef struct smc_ctx smc_ctx;

/* Device bytes the context needs for `cfg` (0 on an invalid config). */
size_t smc_workspace_bytes(const smc_config *cfg);

/* Create a context.  d_workspace: caller-owned device memory of at least
 * smc_workspace_bytes(cfg) bytes, 256-byte aligned; cuda_stream: a
 * cudaStream_t (NULL = legacy default stream).  The context allocates no
 * device memory; it takes a small pinned host buffer mapped into the device's
 * address space (cudaHostAlloc, cudaHostAllocMapped: smc_iterate_host's
 * staging).  The context is ready for smc_set_data; *out is NULL on
 * failure. */
int smc_create(smc_ctx **out, const smc_config *cfg, void *d_workspace, size_t bytes,
               void *cuda_stream);
int smc_destroy(smc_ctx *ctx);

/* Observations.  CV models: `count` rows of (x_obs, y_obs) as float64, row t
 * is Y_t (Algorithm 1).  GMM: `count` float64 data points y_1..y_n.  The data
 * are copied into the workspace. */
int smc_set_data(smc_ctx *ctx, const double *obs, int64_t count, int on_device);

/* Sampler::initialize: t = 0.  CV: X_0 from the prior, weighted by Y_0;
 * GMM: theta from the prior, equal weights, alpha_0 = 0.  Computes the
 * normaliser, ESS and the resample decision of iteration 0. */
int smc_initialize(smc_ctx *ctx);

/* Move queue of the next iteration t (Algorithm 1 / Algorithm 2 "Weight"):
 * CV: gather by the pending ancestors, propagate, add log g(Y_t | X_t);
 * GMM: alpha_t and the incremental weights (alpha_t - alpha_{t-1}) l(theta).
 * Then normaliser, ESS, evidence increment, monitor, resample decision. */
int smc_move(smc_ctx *ctx);

/* Resampling of the current iteration when its ESS test asked for it (or
 * always, when force != 0): fixed-point CDF and ancestor selection by the
 * configured scheme, one cooperative kernel (systematic and stratified:
 * closed-form offspring ranges; multinomial and residual: a histogram of the
 * 24-bit draws; a multinomial or residual context holds 24 MB of workspace
 * for it).  The particle gather happens in the next move/mcmc. */
int smc_resample(smc_ctx *ctx, int force);

/* mcmc queue (Sec. 4.1.3): GMM: the three random-walk Metropolis blocks on
 * mu, log lambda and the weights' log-ratios at alpha_t, then the
 * path-sampling monitor U_t.  CV: nothing. */
int smc_mcmc(smc_ctx *ctx);

/* Sampler::iterate: n iterations of (move, resample, mcmc), replayed from a
 * captured CUDA graph (on a non-default stream, without SMC_FLAG_RECORD):
 * whole chunks of 8 iterations per graph launch, the rest one iteration per
 * launch.  Called while the caller is capturing the context's stream (a
 * particle filter whose one-iteration graph exists, i.e. after one earlier
 * smc_iterate on that stream), the n iterations' kernels are recorded into
 * the caller's graph instead, and the context counts them as run: the caller
 * owns the replays, and an iteration replayed past the observation buffer
 * (max_data rows) raises SMC_E_RANGE on the device and runs nothing.
 * SMC_E_STATE for a capture otherwise (a GMM sampler, SMC_FLAG_RECORD, no
 * graph yet, an invalidated capture). */
int smc_iterate(smc_ctx *ctx, int32_t n);

/* One iteration with host buffers: copies obs_t (CV: 2 float64; may be NULL
 * to use the observation already stored for t) to the device, runs one
 * iteration and copies its record to *h_record.  Returns once the step is
 * done, with the device error word of the step.  SMC_E_ARG past the last
 * observation (or the GMM schedule).  On a non-default stream (and without
 * SMC_FLAG_RECORD) the step is one graph launch: obs_t is placed in the
 * context's mapped pinned staging, which the graph's first kernel reads
 * (and stores, with its float copy, as row t); the record and the error
 * word are written there, and the graph's last kernel then writes the
 * call's sequence number, on which the call waits (spinning on the host,
 * up to a second, then synchronising the stream) instead of synchronising:
 * every kernel of the step has completed when it returns, but a CUDA fault
 * of the step surfaces only at the next call that synchronises.  Otherwise
 * the copies are stream copies and the call synchronises. */
int smc_iterate_host(smc_ctx *ctx, const double *h_obs_t, smc_record *h_record);

/* WeightSet::add_log_weight (Sec. 4.1.6): multiply the current weights by
 * exp(incw_i), i.e. lw_i += incw_i (n_particles values of the context's
 * precision, host or device).  The normaliser L_t, ESS, filtered means and
 * resample decision of the current iteration t are computed again and its
 * record rewritten; the evidence increment L_t is replaced by the new one
 * (log Z_t = log Z_{t-1} + L'_t).  SMC_E_STATE when a resampling of
 * iteration t has already been queued (the current particle system is the
 * pending gather) or before smc_initialize.  A host incw is consumed before
 * the call returns; a device incw must stay valid until the stream reaches
 * the call. */
int smc_add_log_weight(smc_ctx *ctx, const void *incw, int on_device);

/* ESS of the current weights.  h_ess == NULL: no synchronisation. */
int smc_ess(smc_ctx *ctx, double *h_ess);

/* Standard log normalising-constant estimate (sum of L_t), and the
 * path-sampling estimate (GMM).  Synchronise. */
int smc_log_evidence(smc_ctx *ctx, double *h_out);
int smc_path_sampling(smc_ctx *ctx, double *h_out);

/* Current iteration index (the last one completed), -1 before initialize. */
int smc_iteration(const smc_ctx *ctx, int32_t *t);

/* Readers.  Layouts: state is structure-of-arrays, d rows of N values of the
 * context's precision (CV: d = 4, rows x_pos, y_pos, x_vel, y_vel; GMM:
 * d = 3r + 2, rows mu_1..r, lambda_1..r, omega_1..r, log-prior,
 * log-likelihood, followed for the Langevin moves by 3r - 1 rows of the
 * log-likelihood's gradient in (mu, log lambda, log(omega_j / omega_r))).  Log-weights: N values (raw lw_t).  Ancestors: N int32
 * (sorted; valid after a resampling step).  CDF: N uint64 fixed-point
 * inclusive prefix sums (kept only with SMC_FLAG_KEEP_CDF; otherwise
 * smc_read_cdf returns SMC_E_STATE).  Records: the last min(count, available) records in
 * iteration order.  All synchronise. */
int smc_state_dim(const smc_ctx *ctx, int32_t *d);
int smc_read_state(smc_ctx *ctx, void *dst, int on_device);
int smc_read_log_weight(smc_ctx *ctx, void *dst, int on_device);
int smc_read_ancestors(smc_ctx *ctx, int32_t *dst, int on_device);
int smc_read_cdf(smc_ctx *ctx, uint64_t *dst, int on_device);
int smc_read_history(smc_ctx *ctx, smc_record *h_records, int32_t count, int32_t *n_written);

/* Writers: replace the state / log-weights of the current iteration
 * (layouts as above).  smc_write_log_weight then recomputes L_t, ESS, means
 * and the decision as smc_add_log_weight does (with a zero increment), so
 * the evidence increment of iteration t becomes that of the new weights;
 * SMC_E_STATE while a resampling is pending.  Both synchronise. */
int smc_write_state(smc_ctx *ctx, const void *src, int on_device);
int smc_write_log_weight(smc_ctx *ctx, const void *src, int on_device);

/* Checkpoint / resume.  A checkpoint holds the complete sampler state after
 * the last queued call: the device state block (iteration, buffers,
 * normaliser, evidence and path-sampling accumulators, annealing alpha_t,
 * pending-resampling flag), the record ring, the current particle state and
 * log-weights and the pending ancestors.  The random numbers are
 * counter-based, so the checkpoint needs no generator state: restoring it
 * into a context created with the same configuration (and given the same
 * data with smc_set_data first, CV models) continues bit-identically to an
 * uninterrupted run.
 * smc_checkpoint: h_blob == NULL stores the size in *bytes; otherwise
 * *bytes is the capacity of h_blob (SMC_E_ARG and the size in *bytes when
 * too small) and becomes the size written.  Synchronises.
 * smc_restore: SMC_E_ARG when the blob does not match the context's
 * configuration (model, precision, scheme, N, seed, stream id, record ring);
 * SMC_E_STATE when the CV data do not reach the checkpoint's iteration.
 * Not available with SMC_FLAG_RECORD (SMC_E_ARG): the gradient recording is
 * not part of a checkpoint. */
int smc_checkpoint(smc_ctx *ctx, void *h_blob, size_t *bytes);
int smc_restore(smc_ctx *ctx, const void *h_blob, size_t bytes);

/* Tempered log-target of the Gaussian-mixture model and its gradient (the
 * target of the Langevin move, Sec. 5.2 model), at `count` caller-given
 * points in unconstrained coordinates u = (mu_1..r, log lambda_1..r,
 * z_1..r-1), z_j = log(omega_j / omega_r):
 *   gamma(u) = log prior(theta) + alpha l(theta) + sum_j log lambda_j
 *              + sum_j log omega_j   (the last two: log |d theta / d u|),
 * l the log-likelihood of the context's data.  d_u: (3r - 1) rows of
 * `count` values (row-major, the context's precision, device); d_logt:
 * count values; d_grad: (3r - 1) rows of count values (d gamma / d u).  The
 * gradient is the hand-written adjoint through the per-datum log-sum-exp.
 * 0 <= alpha <= 1.  Asynchronous on the context's stream; SMC_E_STATE
 * before smc_set_data; SMC_E_ARG for other models. */
int smc_gmm_log_target(smc_ctx *ctx, const void *d_u, int64_t count, double alpha, void *d_logt, void *d_grad);

/* Gradient of the log-likelihood estimate (CV models, SMC_FLAG_RECORD) with
 * respect to theta = (sd_pos, sd_vel, obs_scale, obs_df) at the context's
 * parameters, after a complete forward run (smc_initialize, then
 * iterations up to the last observation).  The resampling of that run is
 * held fixed (stop-gradient resampling) and the move noise is fixed by its
 * Philox counters; the reverse sweep recomputes the particle trajectory
 * between checkpoints from the recorded ancestors.  grad[3] is 0 for the
 * Gaussian model.  Synchronises. */
int smc_pf_grad(smc_ctx *ctx, double grad[4]);

/* The same recorded run's log-likelihood estimate re-evaluated at another
 * theta with the recorded resampling (for finite differences).
 * Synchronises. */
int smc_pf_replay(smc_ctx *ctx, const double theta[4], double *h_log_evidence);

/* Ancestors chosen at iteration t of a recorded run (N int32; meaningful
 * when that iteration resampled). */
int smc_read_ancestor_history(smc_ctx *ctx, int32_t t, int32_t *dst, int on_device);

/* Profiling hook: two caller-owned CUDA events (cudaEvent_t, created on the
 * context's device; NULL clears) recorded immediately before and after the
 * move kernel inside the iteration graph of smc_iterate, so that their
 * elapsed time is the move kernel's duration within replayed iterations.
 * The graph is captured again at the next smc_iterate; the events then
 * replace the programmatic dependency between the move kernel and the
 * one-pass resampler by an ordinary one.  No counterpart in the paper. */
int smc_set_move_events(smc_ctx *ctx, void *ev_before, void *ev_after);

/* Wait for queued work and return the device error word. */
int smc_sync(smc_ctx *ctx);

const char *smc_error_string(int code);

/* ---- batched form: many independent filters in one launch per kernel ----
 *
 * n_filters constant-velocity particle filters (cfg->model SMC_MODEL_CV or
 * SMC_MODEL_CV_GAUSS, systematic or stratified resampling) that share the
 * model constants, the precision, the threshold and the seed of cfg, each
 * with its own particle count n_particles[b] (1..2^30), its own number of
 * iterations n_iter[b] (= its number of observations) and its own Philox
 * stream cfg->stream_id + b.  Every iteration advances all filters that
 * have observations left with one launch per kernel (a persistent grid over
 * the active filters' tiles); a filter's results equal, bit for bit, a
 * plain context's run on the same stream.  Workspace, stream and error
 * conventions are the plain context's.
 */
typedef struct smc_batch smc_batch;

size_t smc_batch_workspace_bytes(const smc_config *cfg, const int64_t *n_particles, const int32_t *n_iter,
                                 int32_t n_filters);
int smc_batch_create(smc_batch **out, const smc_config *cfg, const int64_t *n_particles, const int32_t *n_iter,
                     int32_t n_filters, void *d_workspace, size_t bytes, void *cuda_stream);
int smc_batch_destroy(smc_batch *b);
/* Philox stream of each filter (stream_ids[f] for filter f, host array of
 * n_filters words; the default is cfg->stream_id + f).  A filter's draws
 * depend only on the key, its stream and the counters (Sec. 3.4: one
 * counter-based stream per unit of work), so a subset of a batch run on
 * another GPU with the same stream ids reproduces those filters exactly.
 * Call before smc_batch_initialize; synchronises. */
int smc_batch_set_streams(smc_batch *b, const uint32_t *stream_ids);
/* observations of filter `filter`: n_iter[filter] rows of (x_obs, y_obs) float64 */
int smc_batch_set_data(smc_batch *b, int32_t filter, const double *obs, int on_device);
/* iteration 0 of every filter (prior draw, weighting by Y_0, resampling) */
int smc_batch_initialize(smc_batch *b);
/* n further iterations of every filter with observations left (CUDA graph
 * replay when the stream is not the legacy default stream) */
int smc_batch_iterate(smc_batch *b, int32_t n);
/* initialize, then iterate until every filter has used all its observations */
int smc_batch_run(smc_batch *b);
/* autotuner: times every launch shape of the persistent kernels -- 1, 2, 3,
 * 4, 6 or 8 resident blocks per SM, each block taking 1, 2 or 4 consecutive
 * tiles per work item -- on the first 10 iterations, keeps the fastest
 * (returned in *blocks_per_sm and *tiles_per_item; either may be NULL) and
 * re-initializes.  The tile (1024 particles, 4 per thread, 256 threads) is
 * not searched: it fixes the reduction order that makes every filter
 * bit-identical to its plain run. */
int smc_batch_tune(smc_batch *b, int32_t *blocks_per_sm, int32_t *tiles_per_item);
/* per-filter log-evidence estimates, n_filters values in caller order */
int smc_batch_log_evidence(smc_batch *b, double *h_out);
int smc_batch_read_history(smc_batch *b, int32_t filter, smc_record *h_records, int32_t count,
                           int32_t *n_written);
/* state of one filter: 4 rows of n_particles[filter] values */
int smc_batch_read_state(smc_batch *b, int32_t filter, void *dst, int on_device);

/* ---- stateless primitives (device pointers, caller's stream) ---- */

/* Philox4x32-10: out[i] = philox(ctr[i], key) for i < n; ctr and out are
 * n x 4 uint32 (row-major), key 2 uint32 (host). */
int smc_philox4x32_10(const uint32_t *d_ctr, const uint32_t key[2], uint32_t *d_out, int64_t n,
                      void *cuda_stream);

/* One shard of a particle filter partitioned over ranks (one GPU each; the
 * paper's MPI module, Sec. 3.1, normalises the weight set across ranks).
 * A filter of n_global particles is split in blocks: this context's
 * n_particles particles are the filter's [offset, offset + n_particles), with
 * those global Philox indices, so every particle evolves as in one context of
 * n_global particles.  CV models and the mixture sampler (with a fixed
 * schedule; Sec. 5.2.5 runs the mixture sampler over MPI ranks), systematic
 * or stratified resampling, without SMC_FLAG_RECORD, _INPLACE or _POST_MEAN;
 * smc_move, smc_resample and smc_iterate refuse a shard (SMC_E_STATE).  One
 * iteration, every rank
 * (the caller runs the collectives between the calls, all buffers device
 * memory on the context's stream):
 *   smc_shard_move(ctx, d_partial)      move + weight; this shard's partial
 *                                       (64 bytes) into d_partial
 *   all-gather of the partials in rank order into d_partials (world x 64 B)
 *   smc_shard_finalize(ctx, d_partials, world)
 *                                       global normaliser, ESS, evidence,
 *                                       means and resampling decision, the
 *                                       same on every rank (record of step t)
 *   then, when the record says resampled:
 *   smc_shard_total(ctx, d_total)       this shard's fixed-point total (uint64)
 *   all-gather of the totals into d_totals (world x uint64)
 *   smc_shard_select(ctx, d_totals, rank, world, d_src, d_range)
 *                                       the global outputs of this shard's
 *                                       particles: d_src[k] = local source of
 *                                       output k (n_global int32), d_range =
 *                                       [k_lo, k_hi) (2 int64)
 *   smc_shard_pack(ctx, d_src, k_lo, k_hi - k_lo, d_send)
 *                                       the copies' states (4 values each, the
 *                                       context's precision) in output order
 *   all-to-all: the copies for output slots [o_d, o_d + n_d) go to rank d
 *   smc_shard_unpack(ctx, d_recv)       the received n_particles copies (output
 *                                       order = slot order) become the shard's
 *                                       particles, log-weights -log n_global
 *   the mixture sampler then (iterations t >= 1):
 *   smc_shard_mcmc(ctx, d_partial)      the Metropolis / Langevin moves of the
 *                                       shard's particles; its partial (64 B,
 *                                       with the shard's accepted-move counts)
 *   all-gather of the partials into d_partials
 *   smc_shard_mcmc_finalize(ctx, d_partials, world)
 *                                       path-sampling integrand U_t and
 *                                       acceptance rates of the whole sampler
 * For the mixture sampler smc_shard_move is the reweighting at alpha_t (and
 * at iteration 0 the prior draws), smc_shard_finalize its normaliser and
 * decision.  The pack and unpack carry every state row (d values a copy).
 * smc_shard_configure marks the context as a shard (before smc_initialize,
 * which then only resets the state: iteration 0 is a smc_shard_move like the
 * others).  Errors: SMC_E_ARG for an unsupported configuration or
 * inconsistent sizes, SMC_E_STATE for a call on a context that is not a
 * shard or out of order. */
int smc_shard_configure(smc_ctx *ctx, int64_t n_global, int64_t offset);
int smc_shard_move(smc_ctx *ctx, void *d_partial);
int smc_shard_finalize(smc_ctx *ctx, const void *d_partials, int32_t world);
int smc_shard_total(smc_ctx *ctx, uint64_t *d_total);
int smc_shard_select(smc_ctx *ctx, const uint64_t *d_totals, int32_t rank, int32_t world, int32_t *d_src,
                     int64_t *d_range);
int smc_shard_pack(smc_ctx *ctx, const int32_t *d_src, int64_t k_lo, int64_t count, void *d_send);
int smc_shard_unpack(smc_ctx *ctx, const void *d_recv);
int smc_shard_mcmc(smc_ctx *ctx, void *d_partial);
int smc_shard_mcmc_finalize(smc_ctx *ctx, const void *d_partials, int32_t world);

/* Measurement: issue rate of the special-function (MUFU) pipe of the current
 * device, the roofline denominator of the likelihood-bound GMM moves (no
 * counterpart in the paper).  One launch of blocks_per_sm x SMs blocks of 256
 * threads, each running 8 independent chains of MUFU approximations for
 * iters rounds -- kind 0: alternating ex2 / lg2, 1: ex2 alone, 2: lg2
 * alone -- after one warm-up launch; *ops_per_s receives MUFU operations per
 * second and *ms the timed launch's duration (CUDA events on a private
 * stream).  Allocates a small buffer; returns SMC_E_ARG for a bad argument
 * and SMC_E_CUDA if a CUDA call fails. */
int smc_mufu_rate(int32_t kind, int32_t blocks_per_sm, int32_t iters, double *ops_per_s, double *ms);

/* Failure detection (bounded device waits).  Every wait of a kernel on
 * another block (the grid barriers of the cooperative resampling kernels, the
 * bulk-copy wait of the GMM kernels) polls at most a fixed number of times,
 * then raises SMC_E_TIMEOUT in the context's device error word and returns
 * instead of hanging.  smc_set_wait_limit sets that number of polls on the
 * current device (default 2^24, about a second; 0 restores the default); it
 * applies to later launches of every context on the device.
 * smc_wait_selftest queues on the context's stream one block that waits at
 * the grid barrier for a second block that does not exist: after the limit
 * the wait gives up, the next synchronising call returns SMC_E_TIMEOUT, and
 * nothing but the error word changes (smc_restore of an earlier checkpoint,
 * or smc_initialize, clears it).  No failure detection in the paper; this is
 * the device half of the host-side status codes. */
int smc_set_wait_limit(uint32_t polls);
int smc_wait_selftest(smc_ctx *ctx);

/* Systematic resampling straight from N float32 log-weights (device) into N
 * int32 ancestors (device), for callers that cannot allocate device memory:
 * code running inside a region that a framework's allocator owns, a loop
 * that must not pay cudaMalloc's implicit synchronisation, or a deployment
 * with a fixed memory budget.  The paper has no counterpart; it is an
 * allocation-free variant of the resampling step of this library.
 * The result equals smc_resample's for a context with the same seed,
 * stream_id and iteration t whose current log-weights are d_log_weight
 * (ancestors sorted, the copy_from convention of the context API).
 * Scratch: one fixed array inside the library, about 17 KB on every GPU that
 * loads it, kept until the process exits; N above 2^22 is rejected with
 * SMC_E_ARG.  The first call on each device looks up the array's device
 * address; make that first call outside any CUDA graph capture.  Every call
 * on a device shares the array and leaves its contents behind (each call
 * clears what it needs first), so calls that overlap on the GPU (other
 * streams, other threads) race: serialise them.  d_log_weight must be
 * 16-byte aligned.  Asynchronous on cuda_stream: a NaN log-weight, or a maximum
 * that is not finite (all -inf), makes the call write nothing and leaves
 * SMC_E_NONFINITE in the array's status word, which
 * smc_resample_noalloc_status reads.  The cached device address is that of
 * the device's primary context: after cudaDeviceReset the process must not
 * call this entry point again. */
int smc_resample_systematic_noalloc(const float *d_log_weight, int64_t n, uint64_t seed, uint32_t stream_id,
                                    int32_t t, int32_t *d_ancestors, void *cuda_stream);

/* Status of the last smc_resample_systematic_noalloc call queued on this
 * device: waits for cuda_stream, then stores SMC_OK or SMC_E_NONFINITE
 * (nothing was written to d_ancestors) in *h_status.  A 4-byte copy from the
 * library's array into a local variable; allocates nothing.  Returns
 * SMC_E_CUDA if the copy or the wait fails. */
int smc_resample_noalloc_status(void *cuda_stream, int32_t *h_status);

#ifdef __cplusplus
}
#endif

#endif /* SMC_H */
