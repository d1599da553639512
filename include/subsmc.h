/*
 * subsmc.h -- C ABI of the GB300 (sm_103a) library for likelihood-annealed subsampling SMC
 * (Gunawan, Dang, Quiroz, Kohn & Tran, arXiv:1805.03317).
 *
 * Conventions for every entry point:
 *   - Return value: SMC_OK (0) or a negative smc_status. Nothing throws across the ABI.
 *     smc_last_error() returns a NUL-terminated description of the last failure on a context.
 *   - Pointers marked "device" are CUDA device pointers; "host" are ordinary host pointers;
 *     "any" accepts either (the library copies with cudaMemcpyDefault, so host memory may be
 *     pageable or pinned). The caller owns every buffer it passes; the library owns the context
 *     and all memory it allocates, and frees it in smc_free().
 *   - All GPU work is enqueued on the stream given to smc_init(). Entry points that return host
 *     scalars synchronise that stream before returning.
 *   - Particle state precision ("state type"): double when the problem's x_dtype is SMC_F64,
 *     float otherwise. theta, gradients and caller-provided particle buffers use it. Control-variate
 *     moments, log weights, the temperature, the log marginal likelihood and MH log ratios are FP64.
 *   - Notation follows the paper: n rows, p parameters, N particles (the paper's M), subsample
 *     size m, G blocks of u, L leapfrog steps, temperature a in [0,1].
 */
#ifndef SUBSMC_H
#define SUBSMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct smc_ctx smc_ctx;

typedef enum {
  SMC_OK = 0,
  SMC_ERR_ARG = -1,       /* invalid argument, shape or layout                                  */
  SMC_ERR_CUDA = -2,      /* a CUDA runtime call failed (message in smc_last_error)            */
  SMC_ERR_NONFINITE = -3, /* a non-finite value appeared where the method needs a finite one    */
  SMC_ERR_TIMEOUT = -4,   /* an iteration cap in a device loop was reached                       */
  SMC_ERR_OOM = -5,       /* device allocation failed                                           */
  SMC_ERR_STATE = -6      /* call out of order (e.g. a stage step before smc_init finished)      */
} smc_status;

/* Per-row likelihood families l_k(theta) = log p(y_k | x_k' theta) (Sec. 3.1, Eq. likelihood).
 * Logistic: Sec. 4.2 (Experiment 1); Poisson with log link and Student-t regression (errors
 * t_nu with scale s): Sec. 4.3 (Experiment 2); Gaussian response with known sd and probit: used by
 * the synthetic workloads. */
typedef enum {
  SMC_LOGISTIC = 0,
  SMC_PROBIT = 1,
  SMC_POISSON = 2,
  SMC_GAUSSIAN = 3,
  SMC_STUDENT_T = 4
} smc_family;

/* Storage type of the covariate matrix X. */
typedef enum { SMC_F64 = 0, SMC_F32 = 1, SMC_BF16 = 2 } smc_dtype;

/* The paper's problem statement (Sec. 2.1 and Sec. 3.1): independent rows (x_k, y_k), a GLM
 * likelihood, and a prior p(theta), here a diagonal Gaussian N(prior_mean, diag(prior_var)). */
typedef struct {
  int32_t family;            /* smc_family                                                        */
  int64_t n;                 /* number of rows, >= 1                                              */
  int32_t p;                 /* number of parameters, 1 <= p <= 126                              */
  const void *X;             /* device, row-major [n, x_ld], element type x_dtype. Read only     */
                             /* inside smc_init (the library keeps its own packed copy).         */
  int32_t x_dtype;           /* smc_dtype                                                         */
  int64_t x_ld;              /* row stride of X in elements, >= p                                 */
  const void *y;             /* device [n]: double when x_dtype == SMC_F64, else float.           */
                             /* Read only inside smc_init.                                        */
  const double *prior_mean;  /* host [p]                                                          */
  const double *prior_var;   /* host [p], every entry > 0                                         */
  double noise_sigma;        /* Gaussian family: known response sd (> 0); Student-t: the error    */
                             /* scale s (> 0); ignored otherwise                                  */
  double dof;                /* Student-t: degrees of freedom nu (> 0; the paper's nu = 5);      */
                             /* ignored otherwise                                                 */
} smc_problem;

/* Run settings. The paper's tuning knobs (Sec. 3.4, Sec. 4.1): M particles, m, G, the ESS target,
 * the leapfrog step and count; R moves per stage is an argument of smc_move(). */
typedef struct {
  int32_t N;                 /* particles (the paper's M), 1 <= N < 2^23                          */
  int32_t m;                 /* subsample size, >= 1                                              */
  int32_t G;                 /* blocks of u for the block pseudo-marginal update, 1 <= G <= m     */
  int32_t L;                 /* leapfrog steps per HMC move, >= 1                                 */
  double ess_frac;           /* ESS target as a fraction of N, in (0, 1]                          */
  uint64_t seed;             /* key of the Philox4x32-10 streams                                  */
  int32_t search_k;          /* K of the K-ary temperature search (2 = bisection); 0 -> 16        */
  int32_t search_rounds;     /* refinement rounds; 0 -> 10                                        */
  double eps0;               /* initial leapfrog step; <= 0 -> 0.5 * p^(-1/4)                     */
  int32_t tile_hint;         /* estimator tile: 0 = automatic, k >= 1 = compiled tile k-1         */
  int32_t hmc_kernel;        /* HMC trajectory kernel: 0 = automatic (rows resident in shared      */
                             /* memory when they fit, else streamed), 1 = streamed, k >= 2 =      */
                             /* resident tile k-2                                                  */
  int32_t cv_kernel;         /* control-variate moments: 0 = automatic (tensor cores, tcgen05,     */
                             /* for BF16 storage with p <= 128; SIMT otherwise), 1 = SIMT          */
  int32_t cv_order;          /* Taylor order of the control variates: 0 or 2 = second order (Sec. */
                             /* 3.2), 1 = first order (q_k = l_k + grad l_k'delta at theta_bar)    */
  int32_t cv_centre;         /* 0 = fixed centre (theta_bar given, else the posterior mode);       */
                             /* 1 = re-centred every stage as in Alg. 2 (d): after the reweighting */
                             /* theta_bar = sum_i W_i theta_i, then A, B, C, the row constants and */
                             /* every particle's cached l_hat, sigma2_hat are recomputed there     */
                             /* before resampling and the moves;                                   */
                             /* 2 = re-centred at the start of every stage, at the weighted mean   */
                             /* of the current cloud, and the cache recomputed before reweighting. */
                             /* Both are stream-ordered (no host sync; graph stages carry them)    */
  int32_t full_data;         /* 1: the comparison method of Sec. 4, full-data SMC: the cache holds  */
                             /* the exact l(theta) (sigma2 = 0), smc_move runs HMC on the exact    */
                             /* tempered posterior with loglik_full forces (no u update); BF16     */
                             /* storage and p <= 64 only. 0: subsampling SMC                       */
  int32_t resampling;        /* 0 = systematic (one uniform per stage); 1 = multinomial, one       */
                             /* uniform per offspring (the paper's scheme, Sec. 2.2). Both act on  */
                             /* integer weights floor(W_i 2^40) and are exact                      */
  int32_t grid_points;       /* 0 = the K-ary bracket search for the next temperature; S >= 2 =    */
                             /* the paper's grid rule (Sec. 2.3): the increment is the point of a   */
                             /* geometric grid of S values over [(1-a) 10^-E, 1-a] whose ESS is    */
                             /* closest to ess_frac * N (ties: the smaller increment)              */
  double grid_decades;       /* E of the grid, > 0; 0 -> 16                                        */
  int32_t theta_move;        /* Markov move of theta given u (Algorithm 1 step 2, Sec. 4.2's         */
                             /* comparison): 0 = HMC with L leapfrog steps (L = 1 is MALA);         */
                             /* 1 = random-walk Metropolis, theta* = theta + eps * Lc z with Sigma  */
                             /* = Lc Lc' the particle covariance, one estimator pass per move, the  */
                             /* step size steered to acceptance 0.234 (HMC: 0.65). Subsampling only */
  double eps_jitter;         /* HMC: particle i's trajectory uses step eps * U_i, U_i uniform on    */
                             /* [1 - j, 1 + j] (second word of its theta-MH Philox block); random   */
                             /* steps break near-periodic trajectories of a fixed eps L (Neal 2011, */
                             /* cited in Sec. 1). j < 0.9; 0 -> 0.3; negative -> a fixed step       */
  int32_t shard_base;        /* Particle sharding (see "Particle shards" below). shard_count = 0:   */
  int32_t shard_count;       /* off. Otherwise smc_move moves only particles [shard_base,           */
                             /* shard_base + shard_count) of the N, with their global indices in   */
                             /* every random stream, and leaves the step-size update to            */
                             /* smc_finish_moves. Needs cv_centre = 0, full_data = 0               */
} smc_config;

/* ------------------------------------------------------------------------------------------- */
/* Lifetime                                                                                     */
/* ------------------------------------------------------------------------------------------- */

/* Create a context (Algorithm 2 step 1). Packs X and y into the library's row layout, sets the
 * control-variate centre theta_bar (host [p]; NULL = the full-data posterior mode, found by Newton's
 * method on the device), computes the moments A, B, C at theta_bar (Sec. 3.2), draws theta ~ p(theta)
 * and u ~ p(u) for every particle, sets W = 1/N and caches l_hat, sigma2_hat per particle.
 * stream: a cudaStream_t (NULL = legacy default stream). On failure *out is NULL. */
int smc_init(smc_ctx **out, const smc_problem *prob, const smc_config *cfg,
             const double *theta_bar, void *stream);

/* Release the context and all library-owned device memory. NULL is allowed. */
int smc_free(smc_ctx *ctx);

/* Description of the last error on ctx (or of the last failed smc_init when ctx is NULL). */
const char *smc_last_error(const smc_ctx *ctx);

/* ------------------------------------------------------------------------------------------- */
/* One SMC stage: smc_reweight, smc_resample, smc_move (Algorithm 2 steps (a)-(f))               */
/* ------------------------------------------------------------------------------------------- */

/* Steps (a)-(d): advance the stage counter; choose the next temperature a_s so that the ESS of the
 * new weights stays at ess_frac*N (Sec. 2.2; K-ary refinement of a bracket, Algorithm 2 (b); or,
 * with smc_config.grid_points > 0, the grid point whose ESS is closest to ess_frac*N, Sec. 2.3);
 * reweight with w_i = W_i exp((a_s - a_{s-1}) l_hat_i - (a_s^2 - a_{s-1}^2) sigma2_hat_i / 2)
 * (Sec. 3.3) and normalise in FP64; accumulate log Z_s/Z_{s-1} (Sec. 3.5); form the weighted
 * particle covariance Sigma and its Cholesky factor for the HMC mass matrix H = Sigma^{-1}
 * (jitter 1e-10 tr(Sigma)/p, x10 per retry, up to 12 retries; if Sigma stays singular, e.g. for a
 * single particle, the previous stage's mass matrix is kept; at the start it is the prior covariance).
 * With smc_config.cv_centre = 1 the control variates then move to the reweighted particle mean
 * (Algorithm 2 (d)); with cv_centre = 2 they move to the current weighted mean before the
 * reweighting. Either way A, B, C, the row constants and every particle's cached l_hat and
 * sigma2_hat are recomputed, stream-ordered (no host synchronisation). The temperature search and
 * the reweighting run as one launch whose blocks wait for each other between phases (at most 152
 * blocks, all resident at once); a wait that does not end within about 2 s is reported as
 * SMC_ERR_TIMEOUT, and the context stays usable. Contexts that belong to a batch use one launch
 * per phase instead.
 * Host outputs (any may be NULL): the new temperature, the log-evidence increment and the ESS;
 * with all three NULL nothing synchronises with the host and errors surface at the next read. */
int smc_reweight(smc_ctx *ctx, double *a_next, double *log_z_inc, double *ess);

/* Step (e): resampling with the current weights, carrying theta, u and the cached estimates; then
 * W = 1/N. Weights are quantised to w_i = floor(W_i 2^40), T = sum w_i. Systematic (default): one
 * uniform U per stage, position i = floor((i T + floor(U T)) / N). Multinomial (smc_config.resampling
 * = 1, Sec. 2.2): offspring i's own uniform U_i, position min(floor(U_i T), T - 1). The ancestor is
 * the first particle whose cumulative integer weight exceeds the position, so the ancestors are
 * exact and independent of summation order. ancestors: device [N] int32 or NULL. */
int smc_resample(smc_ctx *ctx, int32_t *ancestors);

/* Step (f): R Markov moves of Algorithm 1 at the current temperature, each a block pseudo-marginal
 * update of u (Eq. acc_prop_u) followed by an HMC move of theta given u (each particle's
 * trajectory with its jittered step, smc_config.eps_jitter) or, with theta_move = 1, a random-walk
 * Metropolis move. Afterwards the step adapts: eps *= clip(exp(theta_acceptance - t), 0.5, 2),
 * t = 0.65 for HMC and 0.234 for the random walk.
 * Host outputs (may be NULL): acceptance rates of the u and theta updates over these R moves. */
int smc_move(smc_ctx *ctx, int32_t R, double *acc_u, double *acc_theta);

/* Step (f) with the number of moves tuned as the paper does (Sec. 3.4, after Buchholz et al.): moves
 * of Algorithm 1 one at a time until the particles have decorrelated from the cloud they started
 * from. After each move rho_c = the correlation across particles of component c between the
 * starting and the current cloud; the moves stop once the ceil(quantile * p)-th smallest rho_c is
 * <= rho_max (the paper: 90% of the components below a threshold), or after R_max moves. The step
 * size then adapts as in smc_move over the moves made. Synchronises with the host after every move
 * (not usable inside smc_stage's graphs).
 * R_max: 1 .. 256 minus the moves already made this stage; rho_max in [-1, 1]; quantile in (0, 1].
 * Host outputs (may be NULL): the number of moves made and the acceptance rates over them. */
int smc_move_adaptive(smc_ctx *ctx, int32_t R_max, double rho_max, double quantile,
                      int32_t *R_used, double *acc_u, double *acc_theta);

/* One whole stage (Algorithm 2 (a)-(f)): smc_reweight, smc_resample and smc_move(R) with no host
 * outputs and no host synchronisation. use_graph = 0 issues the launches one by one. use_graph = 1
 * replays the stage as one CUDA graph: the first call at each of the two particle-buffer parities
 * (resampling alternates between two buffers) and R captures it on a private stream, later calls
 * launch the instantiated graph on the context's stream; the kernels then read the stage index
 * from a device counter, so replays draw the same random numbers as the launch-by-launch path
 * (results are bit-identical). Tracing events are not recorded inside graphs. smc_autotune drops
 * the graphs. Errors inside the graph surface at the next call that reads the device state. */
int smc_stage(smc_ctx *ctx, int32_t R, int32_t use_graph);

/* ------------------------------------------------------------------------------------------- */
/* The subsampled estimator on caller-supplied particles (Sec. 3.2, Eq. difference_estimator_logl)*/
/* ------------------------------------------------------------------------------------------- */

/* For B particles: l_hat_m(theta_b; u_b) and sigma2_hat_m(theta_b; u_b).
 * theta: device [B, p] state type; u: device [B, m] int32 row indices in [0, n);
 * ell, sigma2: device [B] double. Out-of-range indices return SMC_ERR_ARG (checked on device). */
int loglik_est(smc_ctx *ctx, int32_t B, const void *theta, const int32_t *u, double *ell,
               double *sigma2);

/* As loglik_est, plus the gradient of a*l_hat - (a^2/2)*sigma2_hat + log p(theta) for fixed u
 * (the HMC force of Algorithm 1 step 2). grad: device [B, p] state type; ell, sigma2 may be NULL. */
int loglik_grad(smc_ctx *ctx, int32_t B, const void *theta, const int32_t *u, double a,
                void *grad, double *ell, double *sigma2);

/* Full-data log-likelihood, the comparison method of the paper's experiments (Sec. 4): for B
 * particles, ell = sum_{k=1}^{n} l_k(x_k'theta) over all n rows (including the per-row constants)
 * and grad = a * sum_k l'_k(x_k'theta) x_k + grad log p(theta). The linear predictor
 * [B x p] . [p x n] and the gradient contraction [B x n] . [n x p] run on the tensor cores
 * (tcgen05); needs BF16 storage and p <= 64 (else SMC_ERR_ARG). theta: device [B, p] float;
 * ell: device [B] double or NULL; grad: device [B, p] float or NULL. Scratch is context-owned. */
int loglik_full(smc_ctx *ctx, int32_t B, const void *theta, double a, double *ell, void *grad);

/* Forward half of the differentiable estimator: l_hat and sigma2_hat as loglik_est, and for every
 * row j of every particle the increment d_j = l(eta_j) - q_j(theta) and its eta-derivative
 * r_j = l'(eta_j) - l'(eta_bar_j) - l''(eta_bar_j) x_j'(theta - theta_bar) (Sec. 3.2), saved for
 * loglik_bwd. ell, sigma2: device [B] double; d_save, r_save: device [B, m] in the state type
 * (caller-owned). Out-of-range indices return SMC_ERR_ARG. */
int loglik_fwd(smc_ctx *ctx, int32_t B, const void *theta, const int32_t *u, double *ell,
               double *sigma2, void *d_save, void *r_save);

/* Backward half: for upstream gradients g_ell, g_sig2 (device [B] double) of (l_hat, sigma2_hat),
 * grad = g_ell (B + C delta + (n/m) sum_j r_j x_j) + g_sig2 (2 n^2/m^2) sum_j (d_j - dbar) r_j x_j
 * (the exact derivative for fixed u; no prior term), from the values loglik_fwd saved at the same
 * theta and u; rows are gathered again by u. grad: device [B, p] state type. */
int loglik_bwd(smc_ctx *ctx, int32_t B, const void *theta, const int32_t *u, const void *d_save,
               const void *r_save, const double *g_ell, const double *g_sig2, void *grad);

/* ------------------------------------------------------------------------------------------- */
/* State access (for checkpointing, tests and host-resident callers)                             */
/* ------------------------------------------------------------------------------------------- */

/* Copy out theta [N,p] (state type), u [N,m] int32 and normalised weights W [N] double.
 * Pointers are "any" (host or device); each may be NULL. */
int smc_get_particles(smc_ctx *ctx, void *theta, int32_t *u, double *W);

/* Replace the particle cloud. theta [N,p] state type, u [N,m] int32, W [N] double (normalised,
 * or NULL for 1/N); "any" pointers. The cached l_hat, sigma2_hat are recomputed. */
int smc_set_particles(smc_ctx *ctx, const void *theta, const int32_t *u, const double *W);

/* Cached per-particle estimates: ell, sigma2 [N] double; blocks [N, G, 2] double holding, per
 * block of u, (sum of d_j, sum of d_j^2) with d_j = l_{u_j} - q_{u_j}. "any" pointers or NULL. */
int smc_get_cache(smc_ctx *ctx, double *ell, double *sigma2, double *blocks);

/* Control-variate centre and moments (host): theta_bar [p], A, B [p], C [p,p]; any may be NULL. */
int smc_get_centre(smc_ctx *ctx, double *theta_bar, double *A, double *B, double *C);

/* Moments at an arbitrary point theta (host [p]) without changing the context's centre:
 * A = sum_k l_k, B = sum_k grad l_k, C = sum_k hess l_k (host outputs, C row-major [p,p]). */
int smc_cv_moments(smc_ctx *ctx, const double *theta, double *A, double *B, double *C);

/* Mass-matrix inputs of the current stage (host): Sigma [p,p] and its lower Cholesky factor. */
int smc_get_mass(smc_ctx *ctx, double *Sigma, double *chol);

/* Scalars: temperature a, accumulated log Z, stage index, leapfrog step. Host, each may be NULL. */
int smc_get_status(smc_ctx *ctx, double *a, double *log_z, int32_t *stage, double *eps);

/* Overwrite the scalars (stage index, temperature, leapfrog step); log Z is reset to log_z.
 * The cached estimates stay valid (they do not depend on a). */
int smc_set_scalars(smc_ctx *ctx, int32_t stage, double a, double eps, double log_z);

/* Time the estimator's compiled tile shapes on this context's own particles and keep the fastest;
 * then time the HMC trajectory kernels (streamed, and every resident tile that fits) on scratch
 * copies of the particles. The default trajectory kernel (the narrowest resident tile, with the
 * warps per CTA chosen by p and m) is kept unless another one is more than 3% faster, since
 * near-equal kernels trade places by timing noise. The particle state is not changed.
 * Host outputs (may be NULL): the estimator tile as a tile_hint value (>= 1) and the HMC kernel as
 * an hmc_kernel value (1 = streamed, >= 2 = resident tile). */
int smc_autotune(smc_ctx *ctx, int32_t *tile, int32_t *hmc_kernel);

/* Number of kernels this context has launched so far (every launch is counted). */
int64_t smc_launch_count(const smc_ctx *ctx);

/* Tracing. When enabled, every kernel group is bracketed by CUDA events recorded on the context's
 * stream. Groups: 0 estimator (loglik_est / loglik_grad / cache refresh), 1 u-block update,
 * 2 HMC trajectory, 3 temperature search + reweighting, 4 weighted moments + mass matrix,
 * 5 resampling. smc_profile_read synchronises the stream, returns the number of launches and their
 * summed device time in milliseconds for one group, and clears that group's record. */
int smc_profile_enable(smc_ctx *ctx, int32_t on);
int smc_profile_read(smc_ctx *ctx, int32_t group, int64_t *launches, double *total_ms);

/* ------------------------------------------------------------------------------------------- */
/* Particle shards (several processes, one posterior)                                           */
/* ------------------------------------------------------------------------------------------- */

/* The moves of different particles are independent (Sec. 2.1: the method parallelises over the M
 * particles), so R processes (one per GPU) can share one posterior. Each creates a context with
 * the same problem, seed and N, and its own slice [shard_base, shard_base + shard_count) of the
 * particles. The stage's reweighting, moments, mass matrix and resampling then run redundantly on
 * every process over the full arrays (identical inputs give identical temperatures, weights and
 * integer ancestors), while smc_move moves only the slice. Between stages the caller:
 *   1. sums the slices' accept counts (smc_move_accepts) over the processes and passes the totals
 *      to smc_finish_moves (the step-size update of smc_move);
 *   2. gathers every process's slice of theta and of the cached estimates (smc_shard_export) and
 *      writes the full arrays back (smc_shard_import);
 *   3. after smc_resample, hands the u rows of ancestors that lived on another process to the
 *      process that now holds their offspring (smc_shard_gather_u with before_resample = 1 on the
 *      owner, smc_shard_scatter_u on the receiver).
 * u is kept current only inside a process's own slice. The results equal those of one context
 * with all N particles: the same kernels see the same values, and the random streams are indexed
 * by global particle number. */

/* Copy this context's slice of theta [count, p] (state type), the cached l_hat and sigma2_hat
 * [count] and block sums [count, G, 2] (double) to caller buffers ("any"; each may be NULL).
 * Synchronises the stream. SMC_ERR_STATE when the context has no shard. */
int smc_shard_export(smc_ctx *ctx, void *theta, double *ell, double *sigma2, double *blocks);

/* Overwrite theta [N, p], l_hat, sigma2_hat [N] and the block sums [N, G, 2] of all N particles
 * ("any"; each may be NULL) without recomputing the estimates. Synchronises the stream. */
int smc_shard_import(smc_ctx *ctx, const void *theta, const double *ell, const double *sigma2,
                     const double *blocks);

/* rows[k, 0..m) = u of global particle idx[k], k < count; before_resample = 1 reads the indices
 * as they were before the last smc_resample (the ancestors' rows), 0 the current ones.
 * idx, rows: device. Indices outside [0, N) are skipped and reported as SMC_ERR_ARG by the next
 * synchronising call. Stream-ordered. */
int smc_shard_gather_u(smc_ctx *ctx, int32_t count, const int32_t *idx, int32_t *rows,
                       int32_t before_resample);

/* u of global particle idx[k] = rows[k, 0..m), k < count (the current buffer; the cached
 * estimates are not recomputed). idx, rows: device. Stream-ordered. */
int smc_shard_scatter_u(smc_ctx *ctx, int32_t count, const int32_t *idx, const int32_t *rows);

/* Accepted u updates and theta moves since the last smc_move began (this context's particles).
 * Host outputs; synchronises the stream. */
int smc_move_accepts(smc_ctx *ctx, uint64_t *acc_u, uint64_t *acc_theta);

/* The step-size update that smc_move performs for an unsharded context, from accept totals over
 * all processes: eps *= clip(exp(acc_theta / (N R) - t), 0.5, 2) (t = 0.65 for HMC, 0.234 for the
 * random walk). Stream-ordered. */
int smc_finish_moves(smc_ctx *ctx, int32_t R, uint64_t acc_u, uint64_t acc_theta);

/* ------------------------------------------------------------------------------------------- */
/* Resampling without allocation                                                                */
/* ------------------------------------------------------------------------------------------- */

/* Largest N accepted by smc_resample_noalloc. */
#define SMC_NOALLOC_MAX_N 262144

/* The paper has no counterpart to this entry point; it is a service for callers that cannot
 * allocate device memory when they need resampling: code that runs while a CUDA graph is being
 * captured (cudaMalloc is not allowed there), engines whose memory plan is fixed before they start,
 * and hosts that give the GPU a fixed arena and forbid further allocations.
 * It computes the same ancestors as smc_resample on a context configured for systematic
 * resampling (smc_config.resampling = 0), for the same normalised weights, seed and stage (integer
 * weights floor(W_i 2^40), one uniform U from the stage's resampling stream); it does not implement
 * the multinomial scheme. It needs no context and calls no allocator: its scratch is one fixed device array inside this library
 * (SMC_NOALLOC_MAX_N + 2 eight-byte words, about 2 MiB), which every GPU that loads the library
 * holds until the process exits.
 *   N: 1 <= N <= SMC_NOALLOC_MAX_N, otherwise SMC_ERR_ARG (message in smc_last_error(NULL)).
 *   W: device [N] double, normalised weights. ancestors: device [N] int32 output. Caller-owned.
 *   seed, stage: select the uniform exactly as smc_init's seed and the stage index do.
 *   stream: a cudaStream_t (NULL = legacy default stream); the call is asynchronous on it.
 * The first call on each device looks up the scratch array's device address with that device
 * current; make that first call before any stream capture begins. All calls on a device share the
 * one scratch array, so calls whose kernels overlap on the GPU (different streams, no ordering
 * between them) race and may return wrong ancestors: order them on one stream or with events. */
int smc_resample_noalloc(int32_t N, const double *W, uint64_t seed, int32_t stage,
                         int32_t *ancestors, void *stream);

/* ------------------------------------------------------------------------------------------- */
/* Batches of independent posteriors                                                             */
/* ------------------------------------------------------------------------------------------- */

/* Many independent problems (uneven n and p; BF16 storage) stepped together. One context per
 * problem, created as by smc_init with cfgs[q] (all on the same stream; the estimator tile is
 * the narrowest compiled tile that covers the widest row). The trajectories run in groups: each
 * problem goes to the narrowest resident tile (subsample kept in shared memory) that takes its
 * p, m and G, with one, two or four warps per CTA chosen by p and m (one warp for small
 * subsamples, four for large ones), unless cfgs[q].hmc_kernel = 1 asks for the streamed kernel;
 * problems no resident tile takes (p > 40) and random-walk problems form the streamed group.
 * Problems that share a tile and a warp count share one trajectory launch per move. */
typedef struct smc_batch smc_batch;
int smc_batch_init(smc_batch **out, int32_t P, const smc_problem *probs, const smc_config *cfgs,
                   void *stream);
int smc_batch_free(smc_batch *b);
const char *smc_batch_last_error(const smc_batch *b);
/* The context of problem q (owned by the batch: do not free it), for the per-problem calls
 * (smc_get_particles, smc_get_status, loglik_est, ...). */
int smc_batch_context(smc_batch *b, int32_t q, smc_ctx **ctx);
/* The batch's estimator tile as a tile_hint value. */
int smc_batch_tile(const smc_batch *b, int32_t *tile_hint);
/* The trajectory kernel of problem q as an hmc_kernel value (1 = streamed, k >= 2 = resident
 * tile k - 2): a context created with it (and the batch's tile) steps problem q identically. */
int smc_batch_hmc_kernel(const smc_batch *b, int32_t q, int32_t *hmc_kernel);
int64_t smc_batch_launch_count(const smc_batch *b);
/* One stage of every problem (Algorithm 2 (a)-(f)): the temperature search, reweighting,
 * moments, mass matrix and resampling of every problem; when every problem has a fixed centre
 * (cv_centre = 0) they run in shared launches over all problems (each problem with its own
 * block count, so its reductions follow the same order as alone), else per problem side by side
 * on up to 16 side streams forked from and joined back to the batch's stream. Then per move one
 * u-update launch over the particles of all problems and one trajectory launch per group (the
 * groups side by side on the side streams), then the step sizes. use_graph = 1: the whole batch
 * stage is captured once per buffer parity and replayed as one CUDA graph (kernels read the
 * stage index from device counters), with results bit-identical to use_graph = 0 and to stepping
 * each problem alone with the same tiles (smc_batch_tile, smc_batch_hmc_kernel). */
int smc_batch_stage(smc_batch *b, int32_t R, int32_t use_graph);
/* Choose the batch's estimator tile: time the streamed batched trajectory launch over all problems
 * for every compiled tile that covers the widest row (on scratch copies; the state is unchanged)
 * and keep the fastest. The tile serves the u-update launch and the streamed group; the resident
 * groups keep their tiles. Output: the tile as a tile_hint value. */
int smc_batch_autotune(smc_batch *b, int32_t *tile_hint);

#ifdef __cplusplus
}
#endif
#endif /* SUBSMC_H */
