// Internal declarations shared by the kernel translation units and the C ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

namespace subsmc {

// Scalars that live on the device so that a whole stage runs without host round trips.
struct DevState {
  double a;          // current temperature a_s
  double a_prev;     // a_{s-1}
  double log_z;      // accumulated log marginal likelihood estimate (Sec. 3.5)
  double log_z_inc;  // last increment
  double ess;        // ESS at the chosen increment
  double eps;        // leapfrog step
  double lo, hi, dmax, D;  // temperature search bracket
  double best_dist, best_D;  // grid search: the point whose ESS is closest to the target so far
  double lse_new, lse_old, lse_new2;
  int stage;
  int search_done;
  int err;           // bit 0: index out of range, bit 1: non-finite, bit 2: cholesky failed,
                     // bit 3: iteration cap
  int chol_retries;
  unsigned int ticket;       // last-block-done counter for grid reductions
  unsigned int ticket2;
  unsigned long long acc_u, acc_theta;  // accept counters of the current smc_move call
  unsigned long long res_T;  // resampling: total quantised weight
  unsigned long long res_off;
};

enum ErrBits { kErrIndex = 1, kErrNonFinite = 2, kErrChol = 4, kErrCap = 8 };

// Everything a per-particle estimator kernel needs. Pointers to "CT" data use the state type
// (double for FP64 problems, float otherwise).
struct EstArgs {
  // problem
  const void *Xp;  // packed rows [n, S]: x in [0, p), the RowC tail {c0, c1, c2, y} at element Yo
  int64_t n;
  int p, S, Yo, m, G, fam;
  double inv_s2;   // Gaussian family: 1/sigma^2; Student-t: 1/scale^2
  double A;        // sum_k l_k(theta_bar)
  const double *A_dev;  // when set, A is read from here (a centre that moves every stage)
  const void *B_ct, *C_ct, *tb_ct;  // B [p], C [p,p] (symmetric), theta_bar [p]
  const void *mu_ct, *ivar_ct;      // prior mean, 1/prior variance [p]
  double log_prior_const;           // -0.5 * sum log(2 pi v)
  // particles
  int B;                  // number of particles in this launch
  const void *theta;      // [B, p]
  void *theta_out;        // HMC: updated in place (may equal theta)
  const int32_t *u;       // [B, m]
  int32_t *u_mut;         // u-update: indices written here on acceptance
  double *ell, *sig2;     // [B]
  double *blk;            // [B, G, 2] cache of block sums (may be null for the plain estimator)
  double *blk_prop;       // [B, G, 2] scratch: block sums at the HMC end point
  void *grad;             // [B, p] or null
  double a_host;          // temperature when a_from_state == 0
  int a_from_state;
  // moves
  int L;
  const void *Sigma_ct;   // [p, p] mass-matrix inverse (particle covariance)
  const void *Linv_ct;    // [p, p] inverse of the lower Cholesky factor of Sigma
  uint64_t seed;
  int stage, move;
  int32_t *unew;          // [B, maxblk] scratch for proposed block indices
  int maxblk;
  DevState *st;
  // autograd pair: per-row d, r [B, m] (state type), upstream gradients of l_hat, sigma2_hat [B]
  void *dsave, *rsave;
  int stage_dev;          // 1: the stage index comes from st->stage (graph replays), else stage
  int rw;                 // theta move: 0 = HMC (L leapfrog steps), 1 = random-walk Metropolis
  double eps_jitter;      // HMC: particle step sizes uniform on eps [1 - j, 1 + j] (0: fixed)
  int cv_order;           // 1: first-order control variates (row increments without the
                          //    second-order term; C is zero in the state-type copy), else 2
  int i0;                 // moves: global index of the launch's first particle (its B particles
                          //    are i0 .. i0 + B - 1 in every array and random stream)
  const double *g_ell, *g_sig2;
};

// A batch of independent posteriors launched together: per-problem arguments (device array), the
// first global particle of each problem (ascending, offsets[0] = 0), the particle total and the
// per-warp shared-memory stride (the largest over the batch's problems).
struct BatchArgs {
  const EstArgs *probs;
  const int *offsets;
  int nprob, total, wstride;
};

// Tile shape of the estimator: T lanes share one row, each lane holds CPL element slots; NST
// ring stages of streamed rows per warp (resident kernel: unused); warps per CTA; pipe: the
// streamed kernels overlap the gradient partials of one sweep with x'delta of the next (NST >= 3).
struct Tile {
  int T, CPL, NST, warps, pipe;
};

// Launchers, one set per storage type (defined in est_f64.cu, est_f32.cu, est_bf16.cu).
// op: 0 = plain estimator (optionally with gradient), 1 = u-update, 2 = HMC move,
// 3 = estimator saving per-row d, r, 4 = backward from saved d, r.
// Returns a cudaError_t; -1 if the tile id is not compiled for this storage type.
int est_launch_f64(int op, int tile, const EstArgs &a, cudaStream_t s);
int est_launch_f32(int op, int tile, const EstArgs &a, cudaStream_t s);
int est_launch_bf16(int op, int tile, const EstArgs &a, cudaStream_t s);
// Batched u-update (op 1) or streamed HMC move (op 2) over all particles of a batch (BF16 storage);
// per-warp shared-memory bytes of a tile for p covariates (0 for an unknown tile).
int est_launch_batch_bf16(int op, int tile, const BatchArgs &b, cudaStream_t s);
int est_warp_smem_bf16(int tile, int p);
int est_tiles_f64(Tile *out, int cap);
int est_tiles_f32(Tile *out, int cap);
int est_tiles_bf16(Tile *out, int cap);
// HMC trajectory with the subsample resident in shared memory (resident.cuh): one lane per row,
// Tile.CPL covariate slots per lane, Tile.warps warps per CTA. Returns a cudaError_t, -1 for an
// unknown tile, -2 when the plan does not fit (p > CPL or too much shared memory). dry: check
// the fit only.
int res_launch_f64(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry);
int res_launch_f32(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry);
int res_launch_bf16(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry);
int res_tiles_f64(Tile *out, int cap);
int res_tiles_f32(Tile *out, int cap);
int res_tiles_bf16(Tile *out, int cap);
// The resident trajectory over the particles of a batch of problems that share one resident
// tile (BF16 storage): the shared-memory plan is sized by the largest p, m and G among them.
// Returns a cudaError_t, -1 for a tile without a batched form, -2 when the plan does not fit.
int res_launch_batch_bf16(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                          cudaStream_t s, int sms, bool dry);
// Subsample sizes up to which the trajectories run in two-warp CTAs by default (measured on
// GB300: at m <= 512 the per-pass work that every warp repeats outweighs the rows of a warp).
constexpr int kTwoWarpRows = 512;
// Warps per CTA of the default resident tile for p covariates and m subsample rows (measured on
// GB300, 1024 particles per problem): one warp while a warp's rows outweigh the per-pass work
// that every warp repeats (p 9..24 up to m = 400, p > 24 up to m = 160; at p <= 8 two warps
// always do better), two up to m = 512, else four.
inline int res_default_warps(int p, int m) {
  if (p > 8 && m <= (p <= 24 ? 400 : 160)) return 1;
  return m <= kTwoWarpRows ? 2 : 4;
}
// The two-warp (10..16) and one-warp (17..23) tiles of the BF16 table, single problem and batched.
int res_launch_bf16_w2(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry);
int res_launch_batch_bf16_w2(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                             cudaStream_t s, int sms, bool dry);
int res_launch_bf16_w1(int tile, const EstArgs &a, cudaStream_t s, int sms, bool dry);
int res_launch_batch_bf16_w1(int tile, const BatchArgs &b, int p_max, int m_max, int G_max,
                             cudaStream_t s, int sms, bool dry);

// Stage kernels (stage.cu). All return cudaError_t.
int pack_rows(const void *X, int x_dtype, int64_t n, int p, int64_t ld, const void *y, void *Xp,
              int S, int Yo, cudaStream_t s);
// Rewrites the constants c0..c2 in every packed row's tail for the centre tb_ct (state type).
int row_consts(void *Xp, int x_dtype, int64_t n, int p, int S, int Yo, int fam, const void *tb_ct,
               double inv_s2, double nu, cudaStream_t s);
// mode 0: tensor cores (cv_mma.cu) for BF16 storage with p <= 128, SIMT otherwise; mode 1: SIMT.
// sigma2: Gaussian variance or Student-t squared scale; nu: Student-t degrees of freedom.
int cv_moments(const void *Xp, int x_dtype, int64_t n, int p, int S, int Yo, int fam, double sigma2,
               double nu, const double *theta, double *partials, int nblocks, double *A,
               double *B, double *C, int mode, cudaStream_t s);
int cv_moments_mma(const void *Xp, int64_t n, int p, int S, int Yo, int fam, double sigma2,
                   double nu, const double *theta, double *partials, int maxblocks, int *nblocks,
                   cudaStream_t s);
int cv_moments_blocks(int p);
int newton_step(int p, const double *theta, const double *B, const double *C, const double *mu,
                const double *var, double *step, double *work, int *info, cudaStream_t s);
int axpy_vec(int p, const double *x, double t, const double *s, double *out, cudaStream_t st);
int init_particles(int is_f64, int N, int p, int m, int64_t n, uint64_t seed, const double *mu,
                   const double *var, void *theta, int32_t *u, double *logW, double *W,
                   cudaStream_t s);
// grid_points > 0: the paper's grid rule (Sec. 2.3): the increment is the point of a geometric grid
// of grid_points values over [(1 - a) 10^-grid_decades, 1 - a] whose ESS is closest to tau N;
// otherwise the K-ary bracket search of `rounds` rounds.
// one_launch: the whole reweighting as one launch with grid barriers between its phases (its
// blocks must be able to be resident together: not while other such launches may run beside it);
// else one launch per phase.
int reweight(int N, const double *ell, const double *sig2, double *logW, double *W, double tau,
             int K, int rounds, int grid_points, double grid_decades, DevState *st,
             double *partials, int *launches, cudaStream_t s, bool one_launch = true);
int reweight_scratch_doubles();
int weighted_moments(int is_f64, int N, int p, const double *W, const void *theta,
                     double *partials, double *mean, double *Sigma, cudaStream_t s);
int mass_matrix(int is_f64, int p, const double *Sigma_in, double *Sigma, double *chol,
                void *Sigma_ct, void *Linv_ct, double *work, DevState *st, cudaStream_t s);
// stage_dev: 1 = the resampling draw's stage index comes from st->stage (graph replays).
// multinomial: 1 = one uniform per offspring (multinomial), else one per stage (systematic).
int resample(int is_f64, int N, int p, int m, int G, uint64_t seed, int stage, int stage_dev,
             int multinomial,
             const double *W, uint64_t *cum, int32_t *anc, const void *theta, void *theta_out, const int32_t *u,
             int32_t *u_out, const double *ell, double *ell_out, const double *sig2,
             double *sig2_out, const double *blk, double *blk_out, double *logW, double *Wout,
             DevState *st, cudaStream_t s);
// Device stage counter used by graph replays: set it, or advance it by one (single-thread kernels).
int stage_set(DevState *st, int stage, cudaStream_t s);
int stage_advance(DevState *st, cudaStream_t s);
int weights_from(int N, const double *W_in, double *logW, double *W, cudaStream_t s);
// eps *= clip(exp(acceptance - target), 0.5, 2) over the last R moves.
int eps_update(int N, int R, DevState *st, cudaStream_t s, double target = 0.65);

// Candidates per temperature-search round at most (the grid rule evaluates this many per round).
constexpr int kSearchMaxK = 32;
// The stage steps of many problems at once (batches of BF16-stored problems: FP32 states; fixed
// centre). Problem q's arguments for the buffers that are current before the stage's resampling:
struct StageArgs {
  int N, p, m, G, K, last_round, S, multinomial;
  double tau, E, eps_target;
  uint64_t seed;
  DevState *st;
  double *part;                  // the problem's search / moment partials
  const double *ell, *sig2;      // the cached estimates
  double *logW, *W;
  const float *theta;            // the particles
  double *mean, *Sigma_raw, *Sigma, *chol, *work;
  float *Sigma_ct, *Linv_ct;
  uint64_t *cum;
  int32_t *anc;
  float *theta_out;              // resampling writes the other buffer of each pair
  const int32_t *u;
  int32_t *u_out;
  double *ell_out, *sig2_out;
  const double *blk;
  double *blk_out;
};
// Batched launch kinds: each gives problem q the block count of its single-problem launch (so
// every reduction runs in the same order) at blocks off[kind][q] .. off[kind][q + 1] - 1.
enum StageKind { kSkSearch, kSkFinal, kSkMom, kSkSumMean, kSkSumCov, kSkAnc, kSkGather, kSkKinds };
int stage_kind_blocks(int kind, int N, int p);
struct StageBatch {
  int P, max_rounds, max_p;
  const StageArgs *args;  // device [P]
  const int *off;         // device [kSkKinds][P + 1]
  int total[kSkKinds];    // off[kind][P]
};
// Algorithm 2 (a)-(e) for every problem of the batch: the device stage counter advanced, the
// temperature search and reweighting, the weighted moments and mass matrix, resampling into the
// other buffers and the accept counters cleared; launches are counted into *launches.
int stage_batch(const StageBatch &sb, cudaStream_t s, int64_t *launches);
// The step-size update of every problem after R moves.
int eps_update_batch(const StageBatch &sb, int R, cudaStream_t s);
// rho[c] = correlation across the N particles of component c of clouds a and b (state type).
int autocorr(int is_f64, int N, int p, const void *a, const void *b, double *rho, cudaStream_t s);
int to_state_type(int is_f64, int count, const double *src, void *dst, cudaStream_t s);
int round_to_state_type(int is_f64, int count, double *v, cudaStream_t s);

// Full-data log-likelihood on the tensor cores (full_mma.cu), BF16 storage, p <= 64: ell[B] =
// sum_k l_k(theta_i) (+ lconst), grad[B, p] = a grad l + grad log prior (state type, may be null).
// acc: FP64 scratch of full_acc_doubles(); flag: device int set to 1 if a wait timed out.
// a_dev: device temperature (overrides a when not null).
int full_loglik(const void *Xp, int64_t n, int p, int S, int Yo, int fam, double sigma2, double nu,
                const void *theta, int B, double a, const double *a_dev, double lconst,
                const void *mu, const void *ivar, double *acc, int *flag, double *ell, void *grad,
                int sms, cudaStream_t s);
// Full-data HMC move pieces (state type float, p <= 64): momentum and H0; half kick (+ drift);
// Metropolis-Hastings with the exact log-likelihood at the end point.
// full_move_begin also writes each particle's (jittered) step size to eps_out [N], which the
// kicks of its trajectory read.
int full_move_begin(int N, int p, const void *theta, void *thp, void *rho, const void *Linv,
                    const void *Sigma, const void *mu, const void *ivar, const double *ell,
                    uint64_t seed, int stage, int stage_dev, int move, const DevState *st,
                    double *h0, double jitter, float *eps_out, cudaStream_t s);
int full_move_kick(int N, int p, void *thp, void *rho, const void *g, const void *Sigma,
                   const float *eps_i, int drift, cudaStream_t s);
int full_move_accept(int N, int p, void *theta, const void *thp, const void *rho,
                     const void *Sigma, const void *mu, const void *ivar, double *ell,
                     const double *ell_new, const double *h0, uint64_t seed, int stage,
                     int stage_dev, int move, DevState *st, cudaStream_t s);
// Doubles of FP64 scratch (acc) that full_loglik needs for B particles.
int full_acc_doubles(int64_t n, int p, int B, int sms);
// Sum over rows of the theta-free part of the log-density into *out (device double).
int full_loglik_const(const void *Xp, int64_t n, int S, int Yo, int fam, double sigma2, double nu,
                      double *out, cudaStream_t s);

// Message returned by smc_last_error(NULL) (abi.cu).
void set_global_error(const std::string &msg);

}  // namespace subsmc
