/* fsmc -- finite-state-machine multi-chain MCMC on one GPU (B300, sm_103a).
 *
 * C ABI of libfsmc.so.  The library advances m independent Markov chains of one
 * of three samplers whose single-chain transition contains a data-dependent
 * while loop (arXiv 2503.17405):
 *   - elliptical slice sampling (appendix Alg. 8; shrinking bracket loop),
 *   - delayed-rejection Metropolis-Hastings, 3 stages (Sec. 7.1; staged proposals),
 *   - the No-U-Turn sampler, multinomial form (Sec. 7.3; nested doubling loops).
 * Two execution modes implement the two multi-chain programs the paper compares:
 *   FSMC_MODE_FSM   each chain runs as a finite state machine (Sec. 3, Algs. 2/4/5,
 *                   7/9): a launch moves every chain by a fixed budget of states, so
 *                   no chain waits for another;
 *   FSMC_MODE_SYNC  the vectorised sample() of Alg. 6: every iteration of every while
 *                   loop is a grid-wide step, so all chains wait for the slowest one.
 * Both modes consume the same counter-based random numbers, keyed by
 * (chain, sample, draw), so they produce identical samples (Sec. 2.1: sample(x, r)).
 *
 * Conventions
 *   - Every call returns an fsmc_status; nothing aborts or throws across the ABI.
 *     fsmc_last_error() returns a thread-local message for the last failure.
 *   - The caller owns every host buffer it passes; host buffers are only read or
 *     written during the call.  The library owns every device allocation it makes.
 *   - Array layouts are row-major (C order).  Chain index j, sample index i,
 *     coordinate k: samples are [chain][sample][coordinate].
 *   - Streams are cudaStream_t passed as void*; NULL means the legacy default stream.
 *   - Reads are synchronous on the job's stream and widen to double.
 *   - Objects are not thread-safe; use one thread per job (the serving scheduler
 *     created by fsmc_submit serialises its own jobs).
 */
#ifndef FSMC_H_
#define FSMC_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fsmc_engine fsmc_engine;
typedef struct fsmc_target fsmc_target;
typedef struct fsmc_job fsmc_job;

typedef enum fsmc_status {
  FSMC_OK = 0,
  FSMC_EINVAL = -1,   /* invalid argument (sizes, kinds, NULL pointers)          */
  FSMC_ENOMEM = -2,   /* a device or host allocation failed                       */
  FSMC_EADMIT = -3,   /* the job's device footprint exceeds the engine's budget   */
  FSMC_ECUDA = -4,    /* a CUDA runtime call failed; see fsmc_last_error()        */
  FSMC_ETIMEOUT = -5, /* a bounded device-side wait expired (error word set)      */
  FSMC_ESTATE = -6,   /* call not valid in the object's current state             */
  FSMC_EDEVICE = -7,  /* a kernel raised its error word (e.g. shrink cap reached) */
  FSMC_ECANCELED = -8 /* a submitted job was cancelled (fsmc_cancel)              */
} fsmc_status;

/* Targets.  params_host layouts (doubles, row-major):
 *   GAUSS_CONJ  ESS likelihood -|y - x|^2 / (2 s2):  L[d*d] (prior Cholesky), y[d], s2
 *   GP_LOGIT    ESS likelihood -sum_k softplus(-s_k x_k): L[d*d], s[d] (labels in {-1,+1};
 *               fsmc_target_create returns FSMC_EINVAL for any other label value)
 *   FLAT        ESS likelihood f == 1 (prior draws):    L[d*d]
 *   FUNNEL      Neal funnel, v ~ N(0,9), x_i|v ~ N(0,e^v): no params (n_params = 0)
 *   LOGREG      beta ~ N(0,I), y_i ~ Bern(sigmoid(X_i beta)): X[n_data*d], y[n_data]
 *   GAUSS_DIAG  N(mu, diag(sigma^2)):                     mu[d], sigma[d]
 *   MOG         mixture of K = n_data (1..64) Gaussians N(mu_k, S), S = (1 - rho) I + rho 1 1^T
 *               (unit variances, every pair correlated rho; Sec. 7.3's NUTS target), weights w_k:
 *               log pi(x) = log sum_k w_k exp(-(x - mu_k)^T S^-1 (x - mu_k) / 2) (the common
 *               normaliser dropped):                       rho, w[K], mu[K*d]
 *               (-1/(d-1) < rho < 1 and w_k > 0 finite, else FSMC_EINVAL)
 *   GP_REG      ESS likelihood of GP-regression hyperparameters x = (sigma, tau, lambda), d = 3
 *               (Sec. 7.2): log N(y; 0, tau^2 exp(-lambda^2 D) + sigma^2 I) over n = n_data
 *               points (1..512), D the squared distances between inputs:
 *                                                          L[3*3], D[n*n], y[n]
 *               (-inf where the covariance is not positive definite in the job's precision)
 * ESS needs a kind with a prior factor L (GAUSS_CONJ, GP_LOGIT, FLAT, GP_REG); DR, NUTS and
 * SLICE need a full log-density (FUNNEL, LOGREG, GAUSS_DIAG, MOG).  The ESS prior is
 * N(0, L L^T) (Alg. 8).  GP_REG jobs run a chain per warp (the likelihood warp-wide). */
typedef enum fsmc_target_kind {
  FSMC_TGT_GAUSS_CONJ = 0,
  FSMC_TGT_GP_LOGIT = 1,
  FSMC_TGT_FUNNEL = 2,
  FSMC_TGT_LOGREG = 3,
  FSMC_TGT_GAUSS_DIAG = 4,
  FSMC_TGT_FLAT = 5,
  FSMC_TGT_MOG = 6,
  FSMC_TGT_GP_REG = 7
} fsmc_target_kind;

typedef enum fsmc_algo { FSMC_ESS = 0, FSMC_DR = 1, FSMC_NUTS = 2, FSMC_SLICE = 3 } fsmc_algo;

/* FP64: every floating-point operation in double.  FP32: the production mode, single
 * precision throughout (see fsmc_job_create). */
typedef enum fsmc_precision { FSMC_FP64 = 0, FSMC_FP32 = 1 } fsmc_precision;

typedef enum fsmc_mode { FSMC_MODE_FSM = 0, FSMC_MODE_SYNC = 1 } fsmc_mode;

/* Delayed rejection: stage k (k = 0..n_stages-1) proposes y ~ N(x, (scale0 factor^k)^2 I). */
typedef struct fsmc_dr_params {
  int n_stages;  /* 1..3; symmetric: 1..1000 tries                                        */
  double scale0; /* proposal sd of stage 0 (symmetric: of every try)                         */
  double factor; /* stage k uses scale0 * factor^k (ignored when symmetric)                   */
  int symmetric; /* 0: proposals centred at x, general acceptance (Sec. 7.1 reading, above);
                    1: symmetric delayed rejection (Mira 2001, the paper's toy sampler): try k
                    re-centres y_k ~ N(y_{k-1}, scale0^2 I) on the last rejected point and is
                    accepted with min(1, (pi(y_k) - pi*)+ / (pi(x) - pi*)), pi* the largest
                    target value among the rejected tries                                    */
} fsmc_dr_params;

/* Slice sampling (Neal 2003; Fig. 2's slice sampler) on a random line through x: stepping out
 * from an interval of width w placed uniformly around x, at most m - 1 steps in all (Neal's
 * limit, split J = floor(m V) left, m - 1 - J right), then shrinkage.  N_ij counts log-density
 * evaluations (end checks and proposals); the aux output counts proposals. */
typedef struct fsmc_slice_params {
  double w; /* > 0 */
  int m;    /* 1..1000000 */
} fsmc_slice_params;

/* NUTS: leapfrog step eps, at most max_depth doublings, divergence when H - H0 > max_dH. */
typedef struct fsmc_nuts_params {
  double eps;
  int max_depth; /* 1..10 */
  double max_dH;
} fsmc_nuts_params;

/* Launch shape.  Zero fields mean "choose automatically" (the autotuner's cached
 * choice, else a heuristic on the log-density cost). */
typedef struct fsmc_tuning {
  int lanes_per_chain;   /* 1 = chain-per-thread, 8 = four chains per warp (ESS,
                            32 < d <= 256), 16 = two chains per warp (ESS, 32 < d <= 512),
                            32 = chain-per-warp (ESS, NUTS; DR and slice with d > 32),
                            0 = auto                                                      */
  int steps_per_launch;  /* FSM states each chain advances per launch (at most 2^24)       */
  int ring_slots;        /* ESS: pre-generated ellipse directions kept per chain         */
  int threads_per_block; /* 32..256, multiple of 32; GP_REG: the CTA of one chain, 32, 64
                            or 128 (0 auto: more warps when chains are too few to fill
                            the SMs)                                                     */
  int profile_kernels;   /* 1: time every launch with CUDA events (see fsmc_stats)        */
  int generator;         /* ESS directions nu = L z: 0 auto, 1 CUDA cores, 2 tensor cores
                            (tcgen05; FP32 jobs with d <= 256)                            */
  int pipelined;         /* ESS whole runs: 0 auto (on), 1 refill directions for the next
                            round on a second stream while the FSM kernel runs, 2 off      */
  int step_form;         /* FSM step (ablation of Sec. 3 / App. B): 0 auto = 1; 1 bundled
                            and amortised (ESS), condensed single state (DR); 2 the paper's
                            ablations: ESS as the bundled step without amortisation, which
                            calls the log-density in both INIT and SHRINK every step (one of
                            the two calls masked, as vmap runs it); DR with the PROPOSE body
                            unrolled into four states (draw, evaluate, ratio, decide) run one
                            per step (not condensed).
                            Samples and loop counts are the same in both forms; NUTS and
                            submitted (serving) jobs use form 1 only                       */
  int barrier_spin_limit; /* SYNC mode: polls (each ~64 ns of sleep) a grid-barrier wait makes
                            before it gives up with FSMC_ETIMEOUT; 0 = 2^24 (about 1-2 s)   */
  int barrier_test_missing; /* test hook, 0 in production: 1 makes every grid barrier of a
                            SYNC run wait for one block more than the grid has, so that the
                            first wait of every block runs out, the kernel returns and the
                            run fails with FSMC_ETIMEOUT (failure detection without a fault) */
  int sync_form;         /* SYNC mode, ESS jobs (Alg. 6 programs; identical samples): 0 auto = 2;
                            1 sweep: one cooperative kernel, every group walks all its chains each
                            loop iteration and skips those already done, a grid barrier per
                            iteration; 2 list: the chains still in the loop kept in a compacted
                            list shared by the whole grid, a grid barrier per iteration; 3 graph:
                            the list iterations as kernel launches in a CUDA graph whose while
                            loops (conditional nodes) test their conditions on the device; 4
                            resident: the sweep with every chain's state and current direction
                            kept on chip (registers, shared memory) for the whole launch --
                            single-precision GP-logit jobs, 32 lanes per chain, d of 32, 64, 128
                            or 256 (EINVAL otherwise), at most 8 chains per warp of the grid (the
                            run fails with ECUDA beyond).  DR, slice and NUTS jobs run the sweep
                            form                                                               */
} fsmc_tuning;

/* Run statistics (Sec. 4): loop-body counts N_ij and what each mode spent. */
typedef struct fsmc_stats {
  double R_hat;            /* mean_i max_j N_ij / mean_ij N_ij over completed samples    */
  double mean_N;           /* mean_ij N_ij                                               */
  double mean_max_N;       /* mean_i max_j N_ij                                          */
  int64_t samples_done;    /* sum_j t_j                                                  */
  int64_t fsm_steps;       /* FSM states executed, summed over chains                    */
  int64_t sync_iterations; /* SYNC: loop-body iterations executed (sum_i max_j N_ij)     */
  int64_t launches;        /* kernel launches issued by the last run call                */
  double device_ms;        /* device time of the last run call (CUDA events)             */
  int64_t error_word;      /* OR of kernel error bits (1 shrink cap, 2 barrier timeout,
                              4 non-finite log-density treated as -inf)                  */
  /* With tuning.profile_kernels: device time and launch count per kernel class over the
   * last run call.  Class 0: ESS direction generator (nu = L z); 1: FSM step kernel;
   * 2: synchronised kernel; 3: everything else (fills, resets). */
  double kernel_ms[4];
  int64_t kernel_launches[4];
  int64_t columns_generated; /* ESS: (chain, sample) directions produced by class 0       */
} fsmc_stats;

/* ---- engine ----------------------------------------------------------------------
 * Binds the calling thread to `device` and sets the HBM budget for admission
 * (0 = 90% of the free memory at creation).  Errors: EINVAL, ECUDA, ENOMEM. */
fsmc_status fsmc_engine_create(int device, size_t hbm_budget_bytes, fsmc_engine** out);
/* Waits for the serving scheduler, frees every remaining job and target. */
void fsmc_engine_destroy(fsmc_engine* e);
/* Device bytes currently held by targets and jobs of this engine. */
size_t fsmc_engine_bytes_in_use(const fsmc_engine* e);

/* ---- targets (L1: the log-density, Sec. 7 workloads) ------------------------------
 * Copies params_host (n_params doubles, layout above) to the device in both precisions.
 * Errors: EINVAL (kind/d/n_data/n_params mismatch), ENOMEM, ECUDA. */
fsmc_status fsmc_target_create(fsmc_engine* e, fsmc_target_kind kind, int d, int n_data,
                               const double* params_host, size_t n_params, fsmc_target** out);
void fsmc_target_destroy(fsmc_target* t);

/* ---- jobs ------------------------------------------------------------------------------
 * m = n_chains chains of `algo` on target t, n_samples samples each (Alg. 3 / Alg. 7).
 * algo_params: NULL for ESS, const fsmc_dr_params* for DR, const fsmc_nuts_params* for NUTS,
 * const fsmc_slice_params* for SLICE (NULL: w = 1, m = 100).  DR and SLICE: d <= 1024 (a chain per
 * thread up to d = 32, a chain per warp above).
 * x0_host: [n_chains][d] starting points (NULL = zeros), copied to device memory before the
 * call returns (one DMA when the buffer is pinned).  seed keys the random numbers:
 * chain j, sample i, draw q use Philox4x32-10 with key (j, seed_lo) and counter
 * (q, i, tag, seed_hi).  store_samples: 1 keeps every sample on the device
 * (n_chains*n_samples*d values), 0 keeps per-chain running sums of x and x^2 only.
 * Errors: EINVAL (algo/target mismatch, sizes), EADMIT (footprint over the budget; the
 * footprint is reported in fsmc_last_error), ENOMEM, ECUDA. */
fsmc_status fsmc_job_create(fsmc_engine* e, fsmc_target* t, fsmc_algo algo,
                            const void* algo_params, fsmc_precision prec, int64_t n_chains,
                            int64_t n_samples, const double* x0_host, uint64_t seed,
                            int store_samples, fsmc_job** out);
/* Autotuner: picks the launch shape for jobs like (t, algo, algo_params, prec, n_chains) by
 * timing short FSM runs of candidate shapes (lanes per chain, states per launch, ring depth,
 * threads per block, direction generator) on scratch jobs, and returns the fastest in *best
 * (lowest device time per FSM state).  The choice is cached in a text file keyed by device
 * name, sampler, target kind, d, n_data, precision and log2(n_chains): cache_path, else the
 * file named by $FSMC_TUNE_CACHE, else no cache.  Scratch jobs keep moments only and are
 * freed before returning.  Errors: EINVAL, EADMIT, ENOMEM, ECUDA. */
fsmc_status fsmc_autotune(fsmc_engine* e, fsmc_target* t, fsmc_algo algo, const void* algo_params,
                          fsmc_precision prec, int64_t n_chains, const char* cache_path,
                          fsmc_tuning* best);
/* Overrides the launch shape before the first run (EINVAL for unsupported values). */
fsmc_status fsmc_job_set_tuning(fsmc_job* j, const fsmc_tuning* tuning);
fsmc_status fsmc_job_get_tuning(const fsmc_job* j, fsmc_tuning* tuning);
/* Device bytes the job holds. */
size_t fsmc_job_bytes(const fsmc_job* j);

/* Advances the job on `cuda_stream` (cudaStream_t as void*) and returns when done.
 * FSM mode: runs until every chain has n_samples samples, or, if max_fsm_steps > 0, for
 * ceil(max_fsm_steps / steps_per_launch) rounds (a resumable partial run); a round advances
 * every unfinished chain by steps_per_launch states, or fewer when an ESS chain's direction
 * ring runs dry, and by at least one.  Results do not depend on how a run is split into
 * rounds or calls.  SYNC mode runs to completion (max_fsm_steps ignored).
 * A job can be run several times in FSM mode to resume; SYNC requires a fresh or
 * reset job.  Errors: ESTATE, ECUDA, ETIMEOUT, EDEVICE. */
fsmc_status fsmc_job_run(fsmc_job* j, fsmc_mode mode, int64_t max_fsm_steps, void* cuda_stream);
/* Returns the job to its initial state (x0, zero samples) keeping its allocations. */
fsmc_status fsmc_job_reset(fsmc_job* j);
/* Smallest per-chain sample count and whether every chain is finished. */
fsmc_status fsmc_job_progress(fsmc_job* j, int64_t* min_samples, int* done);

/* Copies samples [chain0, chain0+n_chains) x [sample0, sample0+n_samp) to dst_host
 * ([n_chains][n_samp][d] doubles).  ESTATE if the job keeps moments only. */
fsmc_status fsmc_read_samples(fsmc_job* j, int64_t chain0, int64_t n_chains, int64_t sample0,
                              int64_t n_samp, double* dst_host);
/* Same, to device memory in the job's precision (float or double, [n_chains][n_samp][d]). */
fsmc_status fsmc_read_samples_dev(fsmc_job* j, int64_t chain0, int64_t n_chains,
                                  int64_t sample0, int64_t n_samp, void* dst_dev,
                                  void* cuda_stream);
/* counts_host [n_chains][n_samples]: loop-body count N_ij (ESS shrinks, DR stages tried,
 * NUTS leapfrog steps, slice-sampling log-density evaluations); -1 where not yet sampled.
 * aux_host (nullable) [n_chains][n_samples]: NUTS tree depth, slice-sampling proposals (0
 * for ESS and DR).  fsm_steps_host (nullable) [n_chains]: states executed per chain. */
fsmc_status fsmc_read_loop_counts(fsmc_job* j, int32_t* counts_host, int32_t* aux_host,
                                  int64_t* fsm_steps_host);
/* Current state x of every chain, [n_chains][d]. */
fsmc_status fsmc_read_state(fsmc_job* j, double* x_host);
/* Per-chain running sums over kept samples: sum_x, sum_x2 [n_chains][d]; n_kept [n_chains]. */
fsmc_status fsmc_read_moments(fsmc_job* j, double* sum_x, double* sum_x2, int64_t* n_kept);
fsmc_status fsmc_read_stats(fsmc_job* j, fsmc_stats* out);

/* Checkpoint / resume: the full FSM state (state ids, per-chain variables, sample
 * counters, samples and counts).  Pass host_buf = NULL to query *bytes. */
fsmc_status fsmc_job_snapshot(fsmc_job* j, void* host_buf, size_t* bytes);
fsmc_status fsmc_job_restore(fsmc_job* j, const void* host_buf, size_t bytes);
void fsmc_job_destroy(fsmc_job* j);

/* ---- serving: continuous batching ----------------------------------------------------
 * fsmc_submit queues a created job; the engine's scheduler thread admits queued jobs
 * as HBM budget allows (their allocations are made at admission), advances every
 * admitted job by one fused FSM launch per round (all admitted jobs of a kind share
 * one persistent launch), retires finished jobs and frees their memory.  Arrival
 * time is the submit call; latency is completion minus arrival.  SYNC-mode submits run
 * one job at a time to completion (the synchronised baseline).
 * Errors: EINVAL, ESTATE (already submitted or run). */
fsmc_status fsmc_submit(fsmc_engine* e, fsmc_job* j, fsmc_mode mode);
/* *done = 1 when the job has finished; *latency_s = completion - submit (seconds). */
fsmc_status fsmc_poll(fsmc_job* j, int* done, double* latency_s);
/* Asks the scheduler to drop a submitted job: a queued job is never admitted, a running one is
 * retired between rounds (no kernel of it is interrupted).  Returns at once; the job then
 * finishes with status FSMC_ECANCELED (fsmc_poll reports done and returns that status) and its
 * device memory is returned when it is destroyed.  A job that has already finished keeps its
 * result and status.  Errors: EINVAL, ESTATE (the job was not submitted). */
fsmc_status fsmc_cancel(fsmc_job* j);
/* Blocks until every submitted job has finished or timeout_s elapses (ETIMEOUT). */
fsmc_status fsmc_wait_all(fsmc_engine* e, double timeout_s);

/* ---- allocation-free ESS run -------------------------------------------------------------
 * The paper has no counterpart to this entry point.  It serves callers that must not
 * allocate device memory themselves or through this library: code running under a memory
 * planner that owns the whole device budget, a plugin that is handed device buffers but no
 * allocator, or a latency-critical loop in which cudaMalloc's implicit device-wide
 * synchronisation is not acceptable.
 * It runs FP32 elliptical slice sampling in FSM mode to completion -- the same kernels, and
 * the same samples and loop counts, as fsmc_job_run on an FP32 ESS job that stores its
 * samples and uses the CUDA-core direction generator (tuning.generator = 1), for equal
 * inputs, seed and lanes_per_chain (1 or 32).  Every pointer is
 * caller-owned device memory:
 *   L_dev       [d*d] lower Cholesky factor of the prior covariance (read)
 *   vec_dev     [d]   y for GAUSS_CONJ, labels s in {-1,+1} for GP_LOGIT, unused for FLAT (read)
 *   noise_var         GAUSS_CONJ likelihood variance (ignored otherwise)
 *   x0_dev      [n_chains][d] starting points (read)
 *   samples_dev [n_chains][n_samples][d] (written)
 *   counts_dev  [n_chains][n_samples] loop-body counts N_ij (written)
 * Working memory is one 32 MiB array in the library's device image, which every GPU that
 * loads the library holds until the process exits.  A run needs about
 * n_chains * (4 d + 4 W roundup(d, 32) + 48) bytes, with W = 16 ring slots per chain lowered
 * to 8, 4 or 2 when needed to fit; larger runs fail with FSMC_EINVAL and a message stating
 * the limit (n_chains above 32 MiB / 48 bytes is rejected before anything else is sized).
 * The first call on a device looks up the array's device address (cudaGetSymbolAddress)
 * and keeps it for the life of the process, which assumes the device's primary context is
 * not reset (cudaDeviceReset) while the library is loaded.  The call is synchronous: between
 * bursts of launches it copies a device counter to the host and waits on the stream, so it
 * cannot be issued while that stream is being captured into a graph.  It allocates nothing
 * and returns when the run is complete.  All calls on a device share the one array; each
 * call first resets the parts that must start from zero, and calls that overlap on the GPU
 * (from other threads or streams) race with each other.
 * Errors: EINVAL, ECUDA, ETIMEOUT, EDEVICE. */
fsmc_status fsmc_ess_run_static(int target_kind, int d, const float* L_dev, const float* vec_dev,
                                float noise_var, int64_t n_chains, int64_t n_samples,
                                const float* x0_dev, uint64_t seed, int lanes_per_chain,
                                float* samples_dev, int32_t* counts_dev, void* cuda_stream);

const char* fsmc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* FSMC_H_ */
