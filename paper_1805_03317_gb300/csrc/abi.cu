// C ABI of the subsampling-SMC library (declared in include/subsmc.h). Host orchestration only:
// every arithmetic step of the method runs in the kernels of estimator.cuh and stage.cu.
#include <cuda_bf16.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "internal.h"
#include "subsmc.h"

using namespace subsmc;

struct smc_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  // problem
  int fam = 0, x_dtype = 0, is_f64 = 0, esz = 8, S = 0, Sx = 0, Yo = 0, p = 0, cv_kernel = 0;
  int cv_order = 2, cv_centre = 0;  // control-variate order; re-centring (0 none, 1, 2)
  int multinomial = 0;              // resampling scheme (0 systematic, 1 multinomial)
  int rw = 0;                       // theta move: 0 HMC, 1 random-walk Metropolis
  double eps_jitter = 0.3;          // HMC step-size jitter (0: fixed step)
  int grid_points = 0;              // > 0: grid temperature rule with this many points
  double grid_decades = 16.0;
  int shard_base = 0, shard_count = 0;  // shard_count > 0: smc_move moves only this slice
  int64_t n = 0;
  double noise_sigma = 1.0;  // Gaussian sd or Student-t scale (1 for the other families)
  double dof = 0.0;          // Student-t degrees of freedom
  std::vector<double> mu_h, var_h;
  double log_prior_const = 0.0;
  // configuration
  int N = 0, m = 0, G = 0, L = 0, K = 16, rounds = 10, tile = 0;
  int res_tile = -1;  // resident HMC tile, -1 = streamed trajectory kernel
  int sms = 1;
  double tau = 0.5, eps0 = 0.0;
  uint64_t seed = 0;
  // device memory (library-owned)
  std::vector<void *> allocs;
  void *Xp = nullptr;
  double *mu_d = nullptr, *var_d = nullptr;
  void *mu_ct = nullptr, *ivar_ct = nullptr;
  double *tb_d = nullptr, *A_d = nullptr, *B_d = nullptr, *C_d = nullptr;
  void *tb_ct = nullptr, *B_ct = nullptr, *C_ct = nullptr;
  double A_h = 0.0;
  void *theta = nullptr, *theta_alt = nullptr, *grad_scratch = nullptr;
  void *theta0 = nullptr;    // adaptive moves: the cloud at the start of the stage's moves
  double *rho_d = nullptr;   // adaptive moves: componentwise correlations [p]
  int32_t *u = nullptr, *u_alt = nullptr, *unew = nullptr, *anc = nullptr;
  int maxblk = 1;
  double *logW = nullptr, *W = nullptr;
  double *ell = nullptr, *sig2 = nullptr, *blk = nullptr;
  double *ell_alt = nullptr, *sig2_alt = nullptr, *blk_alt = nullptr, *blk_prop = nullptr;
  double *mean_d = nullptr, *Sigma_raw = nullptr, *Sigma_d = nullptr, *chol_d = nullptr;
  double *mass_work = nullptr;
  void *Sigma_ct = nullptr, *Linv_ct = nullptr;
  double *part = nullptr;
  size_t part_bytes = 0;
  uint64_t *cum = nullptr;
  double *scratch_d = nullptr;  // small FP64 scratch (Newton, moments at a point)
  int *info_d = nullptr;
  DevState *st = nullptr;
  // tracing: event pairs per kernel group
  bool prof_on = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof[6];
  std::vector<cudaEvent_t> ev_pool;
  // CUDA graphs of one whole stage (smc_stage), one per buffer parity: the resampling gather
  // alternates between the two particle buffers, so a stage captured at parity q replays correctly
  // only at parity q. Kernels inside them read the stage index from the device counter.
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  int g_R[2] = {0, 0};
  int64_t g_launches[2] = {0, 0};
  int parity = 0;             // 0: theta/u/ell/sig2/blk are the buffers allocated first
  bool capturing = false;     // inside a stream capture: no tracing events
  bool batch_member = false;  // stepped by a batch: its stage kernels may run beside others
  int stage_dev = 0;          // kernels read the stage index from the device counter
  bool dev_stage_synced = false;  // the device counter equals stage
  // full-data comparison (loglik_full): FP64 per-particle accumulators, timeout flag, constant
  double *full_acc = nullptr;
  int64_t full_cap = 0;
  int *full_flag = nullptr;
  double *full_const_d = nullptr;
  double full_const = 0.0;
  bool full_const_ready = false;
  // full-data comparison SMC (smc_config.full_data): the moves use the exact log-likelihood
  int full_data = 0;
  void *fm_thp = nullptr, *fm_rho = nullptr, *fm_g = nullptr;
  double *fm_ell = nullptr, *fm_h0 = nullptr;
  float *fm_eps = nullptr;  // per-particle step sizes of the current move
  cudaGraphExec_t fm_graph = nullptr;
  int64_t fm_launches = 0;
  // host mirrors
  int stage = 0, moves_in_stage = 0;
  int64_t launches = 0;
  std::string err;
};

namespace {

std::string g_init_error;

int fail(smc_ctx *c, int code, const std::string &msg) {
  if (c)
    c->err = msg;
  else
    g_init_error = msg;
  return code;
}

#define CUDA_OK(c, expr)                                                                  \
  do {                                                                                   \
    cudaError_t e_ = (cudaError_t)(expr);                                                \
    if (e_ != cudaSuccess)                                                               \
      return fail(c, SMC_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define LAUNCH(c, expr, nlaunch)                                                        \
  do {                                                                                 \
    int e_ = (expr);                                                                   \
    (c)->launches += (nlaunch);                                                        \
    if (e_ != 0)                                                                       \
      return fail(c, SMC_ERR_CUDA,                                                     \
                  std::string(#expr) + ": " + cudaGetErrorString((cudaError_t)e_));    \
  } while (0)

template <typename P> int dalloc(smc_ctx *c, P **ptr, size_t bytes) {
  void *q = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(&q, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, SMC_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed: " +
                                    cudaGetErrorString(e));
  }
  c->allocs.push_back(q);
  *ptr = reinterpret_cast<P *>(q);
  return SMC_OK;
}

#define ALLOC(c, ptr, bytes)                  \
  do {                                        \
    int r_ = dalloc((c), &(ptr), (bytes));    \
    if (r_ != SMC_OK) return r_;              \
  } while (0)

size_t ct_size(const smc_ctx *c) { return c->is_f64 ? sizeof(double) : sizeof(float); }

int est_tiles(const smc_ctx *c, Tile *out, int cap) {
  if (c->x_dtype == SMC_F64) return est_tiles_f64(out, cap);
  if (c->x_dtype == SMC_F32) return est_tiles_f32(out, cap);
  return est_tiles_bf16(out, cap);
}

cudaEvent_t take_event(smc_ctx *c) {
  if (!c->ev_pool.empty()) {
    cudaEvent_t e = c->ev_pool.back();
    c->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Brackets a kernel group with events when tracing is on.
struct ProfScope {
  smc_ctx *c;
  int group;
  cudaEvent_t a = nullptr;
  ProfScope(smc_ctx *c_, int g) : c(c_), group(g) {
    if (c->prof_on && !c->capturing) {
      a = take_event(c);
      cudaEventRecord(a, c->stream);
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = take_event(c);
      cudaEventRecord(b, c->stream);
      c->prof[group].push_back({a, b});
    }
  }
};

void drop_graphs(smc_ctx *c) {
  for (int q = 0; q < 2; ++q) {
    if (c->gexec[q]) cudaGraphExecDestroy(c->gexec[q]);
    c->gexec[q] = nullptr;
    c->g_R[q] = 0;
  }
}

int res_launch(smc_ctx *c, int tile, const EstArgs &a, bool dry) {
  if (c->x_dtype == SMC_F64) return res_launch_f64(tile, a, c->stream, c->sms, dry);
  if (c->x_dtype == SMC_F32) return res_launch_f32(tile, a, c->stream, c->sms, dry);
  return res_launch_bf16(tile, a, c->stream, c->sms, dry);
}

int res_tiles(const smc_ctx *c, Tile *out, int cap) {
  if (c->x_dtype == SMC_F64) return res_tiles_f64(out, cap);
  if (c->x_dtype == SMC_F32) return res_tiles_f32(out, cap);
  return res_tiles_bf16(out, cap);
}

// HMC trajectory launch: resident rows when chosen, else the streamed kernel.
int hmc_launch(smc_ctx *c, const EstArgs &a) {
  ProfScope ps(c, 2);
  c->launches += 1;
  if (c->res_tile >= 0 && !c->rw) return res_launch(c, c->res_tile, a, false);
  if (c->x_dtype == SMC_F64) return est_launch_f64(2, c->tile, a, c->stream);
  if (c->x_dtype == SMC_F32) return est_launch_f32(2, c->tile, a, c->stream);
  return est_launch_bf16(2, c->tile, a, c->stream);
}

int est_launch(smc_ctx *c, int op, const EstArgs &a) {
  ProfScope ps(c, op >= 3 ? 0 : op);  // the autograd pair counts as estimator work
  c->launches += 1;
  if (c->x_dtype == SMC_F64) return est_launch_f64(op, c->tile, a, c->stream);
  if (c->x_dtype == SMC_F32) return est_launch_f32(op, c->tile, a, c->stream);
  return est_launch_bf16(op, c->tile, a, c->stream);
}

// Smallest compiled tile that covers the packed row (fewest idle slots, then fewest lanes/row).
int default_tile(const smc_ctx *c) {
  Tile t[32];
  const int nt = est_tiles(c, t, 32);
  int best = -1;
  for (int i = 0; i < nt; ++i) {
    if (t[i].T * t[i].CPL < c->Sx) continue;
    if (best < 0) {
      best = i;
      continue;
    }
    const int wi = t[i].T * t[i].CPL, wb = t[best].T * t[best].CPL;
    if (wi < wb || (wi == wb && t[i].T < t[best].T)) best = i;
  }
  return best;
}

EstArgs base_args(const smc_ctx *c);

// Smallest resident tile (4 warps) whose covariate slots cover p and whose plan fits on an SM.
// The tensor-core trajectory kernel (a tile with T = 0) is left to smc_autotune: on the
// workloads measured it is latency-bound and slower than the CUDA-core tiles.
int default_res_tile(smc_ctx *c) {
  Tile t[32];
  const int nt = res_tiles(c, t, 32);
  EstArgs a = base_args(c);
  a.B = c->N;
  auto narrowest = [&](int warps) {  // the narrowest resident tile with `warps` warps that fits
    int best = -1;
    for (int i = 0; i < nt; ++i) {
      if (t[i].T == 0 || t[i].warps != warps || t[i].CPL < c->p) continue;
      if (res_launch(c, i, a, true) != 0) continue;
      if (best < 0 || t[i].CPL < t[best].CPL) best = i;
    }
    return best;
  };
  // fewer warps per CTA for small subsamples (where such a tile is compiled and fits), else four
  int best = -1;
  for (int w = res_default_warps(c->p, c->m); w <= 4 && best < 0; w *= 2) best = narrowest(w);
  return best;
}

EstArgs base_args(const smc_ctx *c) {
  EstArgs a;
  memset(&a, 0, sizeof(a));
  a.Xp = c->Xp;
  a.n = c->n;
  a.p = c->p;
  a.S = c->S;
  a.Yo = c->Yo;
  a.m = c->m;
  a.G = c->G;
  a.fam = c->fam;
  a.inv_s2 = 1.0 / (c->noise_sigma * c->noise_sigma);
  a.A = c->A_h;
  a.A_dev = c->cv_centre ? c->A_d : nullptr;
  a.cv_order = c->cv_order;
  a.rw = c->rw;
  a.eps_jitter = c->eps_jitter;
  a.B_ct = c->B_ct;
  a.C_ct = c->C_ct;
  a.tb_ct = c->tb_ct;
  a.mu_ct = c->mu_ct;
  a.ivar_ct = c->ivar_ct;
  a.log_prior_const = c->log_prior_const;
  a.L = c->L;
  a.Sigma_ct = c->Sigma_ct;
  a.Linv_ct = c->Linv_ct;
  a.seed = c->seed;
  a.stage = c->stage;
  a.unew = c->unew;
  a.maxblk = c->maxblk;
  a.st = c->st;
  return a;
}

int sync_state(smc_ctx *c, DevState *h) {
  CUDA_OK(c, cudaMemcpyAsync(h, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int check_err_bits(smc_ctx *c, const DevState &h) {
  if (h.err == 0) return SMC_OK;
  const int bits = h.err;
  CUDA_OK(c, cudaMemsetAsync(&c->st->err, 0, sizeof(int), c->stream));
  if (bits & kErrIndex) return fail(c, SMC_ERR_ARG, "subsample index outside [0, n)");
  if (bits & kErrChol) return fail(c, SMC_ERR_NONFINITE, "particle covariance not positive definite");
  if (bits & kErrCap) {  // a bounded wait gave up: clear the arrival counters it may have left
    CUDA_OK(c, cudaMemsetAsync(&c->st->ticket, 0, 2 * sizeof(unsigned int), c->stream));
    return fail(c, SMC_ERR_TIMEOUT, "device iteration cap reached");
  }
  return fail(c, SMC_ERR_NONFINITE, "non-finite estimate or weight");
}

// A, B, C at a device point theta (FP64) into A_out/B_out/C_out (device).
int moments_at(smc_ctx *c, const double *theta_d, double *A_out, double *B_out, double *C_out) {
  LAUNCH(c,
         cv_moments(c->Xp, c->x_dtype, c->n, c->p, c->S, c->Yo, c->fam,
                    c->noise_sigma * c->noise_sigma, c->dof, theta_d, c->part,
                    cv_moments_blocks(c->p), A_out, B_out, C_out, c->cv_kernel, c->stream),
         2);
  return SMC_OK;
}

__global__ void k_log_post(int p, const double *theta, const double *mu, const double *var,
                           const double *A, double *out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double lp = *A;
    for (int c = 0; c < p; ++c) {
      const double r = theta[c] - mu[c];
      lp += -0.5 * r * r / var[c];
    }
    *out = lp;
  }
}

__global__ void k_scale(int count, double f, double *v) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < count; e += gridDim.x * blockDim.x)
    v[e] *= f;
}

// A, B, C of the strided subsample of rows 0, stride, 2 stride, .. (the packed rows read with
// stride x their row pitch), scaled by n / n_sub to stand in for the full-data sums.
int moments_strided(smc_ctx *c, const double *theta_d, double *A, int64_t stride) {
  if (stride <= 1) return moments_at(c, theta_d, A, A + 1, A + 1 + c->p);
  const int p = c->p;
  const int64_t ns = (c->n + stride - 1) / stride;
  LAUNCH(c,
         cv_moments(c->Xp, c->x_dtype, ns, p, (int)(c->S * stride), c->Yo, c->fam,
                    c->noise_sigma * c->noise_sigma, c->dof, theta_d, c->part,
                    cv_moments_blocks(p), A, A + 1, A + 1 + p, c->cv_kernel, c->stream),
         2);
  k_scale<<<8, 256, 0, c->stream>>>(1 + p + p * p, (double)c->n / (double)ns, A);
  c->launches += 1;
  CUDA_OK(c, cudaGetLastError());
  return SMC_OK;
}

// Newton's method with step halving on the log posterior whose likelihood sums come from
// moments_strided(stride), from theta_d (updated in place) until the accepted step is below tol
// in every coordinate.
int newton_iterate(smc_ctx *c, double *theta_d, int64_t stride, double tol) {
  const int p = c->p;
  double *A0 = c->scratch_d, *B0 = A0 + 1, *C0 = B0 + p;
  double *A1 = C0 + p * p;
  double *step = A1 + 1 + p + p * p, *cand = step + p, *f_d = cand + p;
  int r = moments_strided(c, theta_d, A0, stride);
  if (r) return r;
  double f, fc;
  std::vector<double> sh(p);
  auto objective = [&](const double *th, const double *A, double *out) -> int {
    k_log_post<<<1, 32, 0, c->stream>>>(p, th, c->mu_d, c->var_d, A, f_d);
    c->launches += 1;
    CUDA_OK(c, cudaGetLastError());
    CUDA_OK(c, cudaMemcpyAsync(out, f_d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    return SMC_OK;
  };
  if ((r = objective(theta_d, A0, &f))) return r;
  for (int it = 0; it < 60; ++it) {
    LAUNCH(c, newton_step(p, theta_d, B0, C0, c->mu_d, c->var_d, step, nullptr, c->info_d,
                          c->stream),
           1);
    int info = 0;
    CUDA_OK(c, cudaMemcpyAsync(&info, c->info_d, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemcpyAsync(sh.data(), step, sizeof(double) * p, cudaMemcpyDeviceToHost,
                               c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    if (info) return fail(c, SMC_ERR_NONFINITE, "Newton step: negative Hessian not positive definite");
    double t = 1.0;
    while (true) {
      LAUNCH(c, axpy_vec(p, theta_d, t, step, cand, c->stream), 1);
      if ((r = moments_strided(c, cand, A1, stride))) return r;
      if ((r = objective(cand, A1, &fc))) return r;
      if (fc >= f || t < 1e-8) break;
      t *= 0.5;
    }
    CUDA_OK(c, cudaMemcpyAsync(theta_d, cand, sizeof(double) * p, cudaMemcpyDeviceToDevice,
                               c->stream));
    CUDA_OK(c, cudaMemcpyAsync(A0, A1, sizeof(double) * (1 + p + p * p),
                               cudaMemcpyDeviceToDevice, c->stream));
    f = fc;
    double mx = 0.0;
    for (int k = 0; k < p; ++k) mx = fmax(mx, fabs(t * sh[k]));
    if (mx < tol) break;
  }
  return SMC_OK;
}

// Posterior mode by Newton's method with step halving (FP64, on the device). With many rows the
// iterations first run on a strided subsample of about kWarmRows rows (its sums scaled by
// n / n_sub), whose mode lies close to the full-data mode, so the full-data iterations (each a
// pass over all n rows) start near it and converge in two or three steps.
constexpr int64_t kWarmRows = 65536;
int newton_map(smc_ctx *c, double *theta_d) {
  CUDA_OK(c, cudaMemcpyAsync(theta_d, c->mu_d, sizeof(double) * c->p, cudaMemcpyDeviceToDevice,
                             c->stream));
  const int64_t stride = c->n / kWarmRows;
  if (stride >= 4 && (int64_t)c->S * stride < (int64_t)1 << 30) {
    const int r = newton_iterate(c, theta_d, stride, 1e-6);
    if (r) return r;
  }
  return newton_iterate(c, theta_d, 1, 1e-10);
}

// Centre theta_bar (device FP64, already in c->tb_d): round to the state type, moments, CT copies
// (C is zero in the copy the kernels read under first-order control variates), and the per-row
// constants at the centre in every packed row's tail. Stream-ordered, no host synchronisation.
int centre_kernels(smc_ctx *c) {
  const int p = c->p;
  LAUNCH(c, round_to_state_type(c->is_f64, p, c->tb_d, c->stream), c->is_f64 ? 0 : 1);
  int r = moments_at(c, c->tb_d, c->A_d, c->B_d, c->C_d);
  if (r) return r;
  LAUNCH(c, to_state_type(c->is_f64, p, c->tb_d, c->tb_ct, c->stream), 1);
  LAUNCH(c, to_state_type(c->is_f64, p, c->B_d, c->B_ct, c->stream), 1);
  if (c->cv_order == 1) {
    CUDA_OK(c, cudaMemsetAsync(c->C_ct, 0, (size_t)p * p * (c->is_f64 ? 8 : 4), c->stream));
  } else {
    LAUNCH(c, to_state_type(c->is_f64, p * p, c->C_d, c->C_ct, c->stream), 1);
  }
  LAUNCH(c,
         row_consts(c->Xp, c->x_dtype, c->n, p, c->S, c->Yo, c->fam, c->tb_ct,
                    1.0 / (c->noise_sigma * c->noise_sigma), c->dof, c->stream),
         1);
  return SMC_OK;
}

int set_centre(smc_ctx *c) {
  int r = centre_kernels(c);
  if (r) return r;
  CUDA_OK(c, cudaMemcpyAsync(&c->A_h, c->A_d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (!isfinite(c->A_h)) return fail(c, SMC_ERR_NONFINITE, "A(theta_bar) is not finite");
  return SMC_OK;
}

// Recompute the per-particle cache (l_hat, sigma2_hat, block sums) at the current particles.
// Full-data log-likelihood (the comparison method): scratch, the theta-free constant (once), and
// one evaluation without host synchronisation.
int full_prepare(smc_ctx *c, int64_t B) {
  if (c->x_dtype != SMC_BF16 || c->p > 64)
    return fail(c, SMC_ERR_ARG, "the full-data kernel needs BF16 storage and p <= 64");
  if (!c->full_const_ready) {
    if (!c->full_flag) ALLOC(c, c->full_flag, 2 * sizeof(double));  // flag, then the constant
    c->full_const_d = reinterpret_cast<double *>(c->full_flag) + 1;
    LAUNCH(c,
           full_loglik_const(c->Xp, c->n, c->S, c->Yo, c->fam, c->noise_sigma * c->noise_sigma,
                             c->dof, c->full_const_d, c->stream),
           1);
    CUDA_OK(c, cudaMemcpyAsync(&c->full_const, c->full_const_d, sizeof(double),
                               cudaMemcpyDeviceToHost, c->stream));
    CUDA_OK(c, cudaMemsetAsync(c->full_flag, 0, sizeof(int), c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    c->full_const_ready = true;
  }
  const int64_t need = full_acc_doubles(c->n, c->p, (int)B, c->sms);
  if (need > c->full_cap) {
    ALLOC(c, c->full_acc, sizeof(double) * (size_t)need);
    c->full_cap = need;
  }
  return SMC_OK;
}

int full_eval(smc_ctx *c, int B, const void *theta, double a, const double *a_dev,
                     double *ell, void *grad) {
  ProfScope ps(c, 0);
  LAUNCH(c,
         full_loglik(c->Xp, c->n, c->p, c->S, c->Yo, c->fam, c->noise_sigma * c->noise_sigma,
                     c->dof, theta, B, a, a_dev, c->full_const, c->mu_ct, c->ivar_ct, c->full_acc,
                     c->full_flag, ell, grad, c->sms, c->stream),
         2);
  return SMC_OK;
}

int full_check_flag(smc_ctx *c) {
  int flag = 0;
  CUDA_OK(c, cudaMemcpyAsync(&flag, c->full_flag, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  if (flag) return fail(c, SMC_ERR_TIMEOUT, "full-data kernel: tensor-core wait timed out");
  return SMC_OK;
}

int refresh_cache(smc_ctx *c) {
  if (c->full_data) {  // the exact log-likelihood; no subsample variance
    int r = full_prepare(c, c->N);
    if (r) return r;
    if ((r = full_eval(c, c->N, c->theta, 1.0, nullptr, c->ell, nullptr))) return r;
    CUDA_OK(c, cudaMemsetAsync(c->sig2, 0, sizeof(double) * c->N, c->stream));
    CUDA_OK(c, cudaMemsetAsync(c->blk, 0, sizeof(double) * c->N * c->G * 2, c->stream));
    return SMC_OK;
  }
  EstArgs a = base_args(c);
  a.B = c->N;
  a.theta = c->theta;
  a.u = c->u;
  a.ell = c->ell;
  a.sig2 = c->sig2;
  a.blk = c->blk;
  a.a_host = 0.0;
  LAUNCH(c, est_launch(c, 0, a), 0);
  return SMC_OK;
}

// Mass matrix from a covariance held in Sigma_raw (device FP64).
int set_mass(smc_ctx *c) {
  LAUNCH(c,
         mass_matrix(c->is_f64, c->p, c->Sigma_raw, c->Sigma_d, c->chol_d, c->Sigma_ct,
                     c->Linv_ct, c->mass_work, c->st, c->stream),
         1);
  return SMC_OK;
}

int init_impl(smc_ctx *c, const smc_problem *P, const smc_config *cfg, const double *theta_bar) {
  const int p = c->p;
  const size_t cts = ct_size(c);
  // packed rows
  ALLOC(c, c->Xp, (size_t)c->n * c->S * c->esz);
  LAUNCH(c, pack_rows(P->X, c->x_dtype, c->n, p, P->x_ld, P->y, c->Xp, c->S, c->Yo, c->stream),
         1);
  // prior
  ALLOC(c, c->mu_d, sizeof(double) * p);
  ALLOC(c, c->var_d, sizeof(double) * p);
  ALLOC(c, c->mu_ct, cts * p);
  ALLOC(c, c->ivar_ct, cts * p);
  std::vector<double> ivar(p);
  for (int k = 0; k < p; ++k) ivar[k] = 1.0 / c->var_h[k];
  CUDA_OK(c, cudaMemcpyAsync(c->mu_d, c->mu_h.data(), sizeof(double) * p, cudaMemcpyHostToDevice,
                             c->stream));
  CUDA_OK(c, cudaMemcpyAsync(c->var_d, c->var_h.data(), sizeof(double) * p,
                             cudaMemcpyHostToDevice, c->stream));
  double *tmp = nullptr;
  ALLOC(c, tmp, sizeof(double) * p);
  CUDA_OK(c, cudaMemcpyAsync(tmp, ivar.data(), sizeof(double) * p, cudaMemcpyHostToDevice,
                             c->stream));
  LAUNCH(c, to_state_type(c->is_f64, p, c->mu_d, c->mu_ct, c->stream), 1);
  LAUNCH(c, to_state_type(c->is_f64, p, tmp, c->ivar_ct, c->stream), 1);
  // scratch
  const int cvw = 1 + p + p * (p + 1) / 2;
  size_t part = (size_t)cv_moments_blocks(p) * cvw * sizeof(double);
  const size_t part_mom = (size_t)152 * p * p * sizeof(double);
  const size_t part_rw = (size_t)reweight_scratch_doubles() * sizeof(double);
  if (part_mom > part) part = part_mom;
  if (part_rw > part) part = part_rw;
  ALLOC(c, c->part, part);
  c->part_bytes = part;
  ALLOC(c, c->scratch_d, sizeof(double) * (2 * (1 + p + p * p) + 3 * p + 8));
  ALLOC(c, c->info_d, sizeof(int) * 4);
  ALLOC(c, c->st, sizeof(DevState));
  CUDA_OK(c, cudaMemsetAsync(c->st, 0, sizeof(DevState), c->stream));
  // control-variate centre and moments
  ALLOC(c, c->tb_d, sizeof(double) * p);
  ALLOC(c, c->A_d, sizeof(double) * (1 + p + p * p));
  c->B_d = c->A_d + 1;
  c->C_d = c->B_d + p;
  ALLOC(c, c->tb_ct, cts * p);
  ALLOC(c, c->B_ct, cts * p);
  ALLOC(c, c->C_ct, cts * p * p);
  int r;
  if (theta_bar) {
    CUDA_OK(c, cudaMemcpyAsync(c->tb_d, theta_bar, sizeof(double) * p, cudaMemcpyHostToDevice,
                               c->stream));
  } else if ((r = newton_map(c, c->tb_d))) {
    return r;
  }
  if ((r = set_centre(c))) return r;
  // particles
  const size_t Np = (size_t)c->N * p, Nm = (size_t)c->N * c->m, NG = (size_t)c->N * c->G * 2;
  if (c->full_data) {  // full-data move buffers: trajectory position, momentum, force, l, H0
    ALLOC(c, c->fm_thp, cts * Np);
    ALLOC(c, c->fm_rho, cts * Np);
    ALLOC(c, c->fm_g, cts * Np);
    ALLOC(c, c->fm_ell, sizeof(double) * c->N);
    ALLOC(c, c->fm_h0, sizeof(double) * c->N);
    ALLOC(c, c->fm_eps, sizeof(float) * c->N);
  }
  ALLOC(c, c->theta, cts * Np);
  ALLOC(c, c->theta_alt, cts * Np);
  ALLOC(c, c->grad_scratch, cts * Np);
  ALLOC(c, c->u, sizeof(int32_t) * Nm);
  ALLOC(c, c->u_alt, sizeof(int32_t) * Nm);
  c->maxblk = (c->m + c->G - 1) / c->G + 1;
  ALLOC(c, c->unew, sizeof(int32_t) * (size_t)c->N * c->maxblk);
  ALLOC(c, c->anc, sizeof(int32_t) * c->N);
  ALLOC(c, c->cum, sizeof(uint64_t) * c->N);
  ALLOC(c, c->logW, sizeof(double) * c->N);
  ALLOC(c, c->W, sizeof(double) * c->N);
  ALLOC(c, c->ell, sizeof(double) * c->N);
  ALLOC(c, c->sig2, sizeof(double) * c->N);
  ALLOC(c, c->ell_alt, sizeof(double) * c->N);
  ALLOC(c, c->sig2_alt, sizeof(double) * c->N);
  ALLOC(c, c->blk, sizeof(double) * NG);
  ALLOC(c, c->blk_alt, sizeof(double) * NG);
  ALLOC(c, c->blk_prop, sizeof(double) * NG);
  ALLOC(c, c->mean_d, sizeof(double) * p);
  ALLOC(c, c->Sigma_raw, sizeof(double) * p * p);
  ALLOC(c, c->Sigma_d, sizeof(double) * p * p);
  ALLOC(c, c->chol_d, sizeof(double) * p * p);
  ALLOC(c, c->mass_work, sizeof(double) * p * p);
  ALLOC(c, c->Sigma_ct, cts * p * p);
  ALLOC(c, c->Linv_ct, cts * p * p);
  LAUNCH(c,
         init_particles(c->is_f64, c->N, p, c->m, c->n, c->seed, c->mu_d, c->var_d, c->theta, c->u,
                        c->logW, c->W, c->stream),
         1);
  if ((r = refresh_cache(c))) return r;
  // initial mass matrix: the prior covariance
  std::vector<double> S0((size_t)p * p, 0.0);
  for (int k = 0; k < p; ++k) S0[(size_t)k * p + k] = c->var_h[k];
  CUDA_OK(c, cudaMemcpyAsync(c->Sigma_raw, S0.data(), sizeof(double) * p * p,
                             cudaMemcpyHostToDevice, c->stream));
  if ((r = set_mass(c))) return r;
  // scalars
  DevState h;
  memset(&h, 0, sizeof(h));
  h.eps = c->eps0 > 0 ? c->eps0 : 0.5 * pow((double)p, -0.25);
  CUDA_OK(c, cudaMemcpyAsync(c->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  if ((r = sync_state(c, &h))) return r;
  (void)cfg;
  return check_err_bits(c, h);
}

}  // namespace

void subsmc::set_global_error(const std::string &msg) { g_init_error = msg; }

extern "C" {

int smc_init(smc_ctx **out, const smc_problem *P, const smc_config *cfg, const double *theta_bar,
             void *stream) {
  if (!out) return fail(nullptr, SMC_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!P || !cfg) return fail(nullptr, SMC_ERR_ARG, "problem or config is NULL");
  if (P->x_dtype < 0 || P->x_dtype > 2) return fail(nullptr, SMC_ERR_ARG, "unknown x_dtype");
  if (P->n < 1 || P->n > 0x7fffffffLL) return fail(nullptr, SMC_ERR_ARG, "n must be in [1, 2^31)");
  if (P->p < 1 || P->p > 126) return fail(nullptr, SMC_ERR_ARG, "p must be in [1, 126]");
  if (P->x_ld < P->p) return fail(nullptr, SMC_ERR_ARG, "x_ld < p");
  if (!P->X || !P->y || !P->prior_mean || !P->prior_var)
    return fail(nullptr, SMC_ERR_ARG, "X, y, prior_mean and prior_var are required");
  for (int k = 0; k < P->p; ++k)
    if (!(P->prior_var[k] > 0) || !isfinite(P->prior_mean[k]))
      return fail(nullptr, SMC_ERR_ARG, "prior variances must be > 0 and means finite");
  if (P->family < SMC_LOGISTIC || P->family > SMC_STUDENT_T)
    return fail(nullptr, SMC_ERR_ARG, "unknown family");
  if ((P->family == SMC_GAUSSIAN || P->family == SMC_STUDENT_T) && !(P->noise_sigma > 0))
    return fail(nullptr, SMC_ERR_ARG, "Gaussian and Student-t families need noise_sigma > 0");
  if (P->family == SMC_STUDENT_T && !(P->dof > 0 && P->dof < 1e6))
    return fail(nullptr, SMC_ERR_ARG, "Student-t family needs dof in (0, 1e6)");
  if (cfg->N < 1 || cfg->N >= (1 << 23)) return fail(nullptr, SMC_ERR_ARG, "N must be in [1, 2^23)");
  if (cfg->m < 1 || cfg->G < 1 || cfg->G > cfg->m)
    return fail(nullptr, SMC_ERR_ARG, "need m >= 1 and 1 <= G <= m");
  if (cfg->L < 1) return fail(nullptr, SMC_ERR_ARG, "L must be >= 1");
  if (!(cfg->ess_frac > 0 && cfg->ess_frac <= 1)) return fail(nullptr, SMC_ERR_ARG, "ess_frac in (0,1]");
  const int K = cfg->search_k ? cfg->search_k : 16, rounds = cfg->search_rounds ? cfg->search_rounds : 10;
  if (K < 2 || K > 32 || rounds < 1 || rounds > 64)
    return fail(nullptr, SMC_ERR_ARG, "search_k in [2, 32], search_rounds in [1, 64]");

  smc_ctx *c = new smc_ctx();
  cudaGetDevice(&c->device);
  c->stream = (cudaStream_t)stream;
  c->fam = P->family;
  c->x_dtype = P->x_dtype;
  c->is_f64 = P->x_dtype == SMC_F64;
  c->esz = P->x_dtype == SMC_F64 ? 8 : (P->x_dtype == SMC_F32 ? 4 : 2);
  // packed row: x, then the tail {c0, c1, c2, y} (four state-type values) from the next 16-byte
  // boundary, stride a multiple of 64 bytes so that a row occupies whole DRAM fetch units
  const int xbytes = ((P->p * c->esz + 15) / 16) * 16;
  const int tbytes = 4 * (c->is_f64 ? 8 : 4);
  c->Yo = xbytes / c->esz;
  c->S = ((xbytes + tbytes + 63) / 64) * 64 / c->esz;
  c->Sx = c->Yo;  // streamed tiles cover the covariate vectors; tails travel separately
  c->n = P->n;
  c->p = P->p;
  c->noise_sigma =
      (P->family == SMC_GAUSSIAN || P->family == SMC_STUDENT_T) ? P->noise_sigma : 1.0;
  c->dof = P->family == SMC_STUDENT_T ? P->dof : 0.0;
  c->mu_h.assign(P->prior_mean, P->prior_mean + P->p);
  c->var_h.assign(P->prior_var, P->prior_var + P->p);
  for (int k = 0; k < P->p; ++k) c->log_prior_const += -0.5 * log(6.283185307179586 * c->var_h[k]);
  c->N = cfg->N;
  c->m = cfg->m;
  c->G = cfg->G;
  c->L = cfg->L;
  c->tau = cfg->ess_frac;
  c->seed = cfg->seed;
  c->K = K;
  c->rounds = rounds;
  c->eps0 = cfg->eps0;
  c->cv_kernel = cfg->cv_kernel == 1 ? 1 : 0;
  if (cfg->cv_order < 0 || cfg->cv_order > 2 || cfg->cv_centre < 0 || cfg->cv_centre > 2) {
    g_init_error = "cv_order must be 0, 1 or 2 and cv_centre 0, 1 or 2";
    delete c;
    return SMC_ERR_ARG;
  }
  if (cfg->resampling < 0 || cfg->resampling > 1 || cfg->grid_points < 0 ||
      cfg->grid_points == 1 || cfg->grid_points > (1 << 16) || !(cfg->grid_decades >= 0.0) ||
      cfg->grid_decades > 300.0) {
    g_init_error = "resampling must be 0 or 1, grid_points 0 or in [2, 65536], grid_decades in "
                   "[0, 300]";
    delete c;
    return SMC_ERR_ARG;
  }
  c->cv_order = cfg->cv_order == 1 ? 1 : 2;
  c->cv_centre = cfg->cv_centre;
  c->multinomial = cfg->resampling;
  if (cfg->theta_move < 0 || cfg->theta_move > 1 || (cfg->theta_move == 1 && cfg->full_data)) {
    g_init_error = "theta_move must be 0 (HMC) or 1 (random walk; subsampling only)";
    delete c;
    return SMC_ERR_ARG;
  }
  c->rw = cfg->theta_move;
  if (!(cfg->eps_jitter < 0.9)) {
    g_init_error = "eps_jitter must be below 0.9 (0: 0.3; negative: a fixed step size)";
    delete c;
    return SMC_ERR_ARG;
  }
  c->eps_jitter = cfg->eps_jitter == 0.0 ? 0.3 : (cfg->eps_jitter < 0.0 ? 0.0 : cfg->eps_jitter);
  c->grid_points = cfg->grid_points;
  c->grid_decades = cfg->grid_decades > 0.0 ? cfg->grid_decades : 16.0;
  if (cfg->shard_count < 0 || cfg->shard_base < 0 ||
      (cfg->shard_count > 0 && (int64_t)cfg->shard_base + cfg->shard_count > cfg->N) ||
      (cfg->shard_count > 0 && (cfg->cv_centre != 0 || cfg->full_data))) {
    g_init_error = "shard: need 0 <= shard_base, shard_base + shard_count <= N, cv_centre = 0 and "
                   "full_data = 0";
    delete c;
    return SMC_ERR_ARG;
  }
  c->shard_base = cfg->shard_base;
  c->shard_count = cfg->shard_count;
  c->full_data = cfg->full_data ? 1 : 0;
  if (c->full_data && (P->x_dtype != SMC_BF16 || P->p > 64)) {
    g_init_error = "full_data needs BF16 storage and p <= 64";
    delete c;
    return SMC_ERR_ARG;
  }
  c->tile = cfg->tile_hint > 0 ? cfg->tile_hint - 1 : default_tile(c);
  Tile tl[32];
  const int nt = est_tiles(c, tl, 32);
  if (c->tile < 0 || c->tile >= nt || tl[c->tile].T * tl[c->tile].CPL < c->Sx) {
    g_init_error = "no compiled tile covers this row width";
    delete c;
    return SMC_ERR_ARG;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (c->sms < 1) c->sms = 1;
  const int r = init_impl(c, P, cfg, theta_bar);
  if (r != SMC_OK) {
    g_init_error = c->err;
    smc_free(c);
    return r;
  }
  if (cfg->hmc_kernel == 0) {
    c->res_tile = default_res_tile(c);
  } else if (cfg->hmc_kernel >= 2) {
    Tile tr[32];
    const int nr = res_tiles(c, tr, 32);
    EstArgs a = base_args(c);
    a.B = c->N;
    if (cfg->hmc_kernel - 2 >= nr || res_launch(c, cfg->hmc_kernel - 2, a, true) != 0) {
      g_init_error = "resident HMC tile not compiled or does not fit this problem";
      smc_free(c);
      return SMC_ERR_ARG;
    }
    c->res_tile = cfg->hmc_kernel - 2;
  }
  *out = c;
  return SMC_OK;
}

int smc_free(smc_ctx *c) {
  if (!c) return SMC_OK;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  if (c->fm_graph) cudaGraphExecDestroy(c->fm_graph);
  for (void *q : c->allocs) cudaFree(q);
  for (auto &v : c->prof)
    for (auto &pr : v) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
  delete c;
  return SMC_OK;
}

const char *smc_last_error(const smc_ctx *c) {
  return c ? c->err.c_str() : g_init_error.c_str();
}

// Re-centre the control variates at the weighted particle mean in c->mean_d (Alg. 2 (d)): A, B,
// C and the row constants there, then every particle's l_hat, sigma2_hat and block sums under the
// new control variates, so that the next comparisons of estimates use one estimator. A non-finite
// A surfaces through the estimates' error bits. Stream-ordered, no host synchronisation.
static int recentre(smc_ctx *c) {
  CUDA_OK(c, cudaMemcpyAsync(c->tb_d, c->mean_d, sizeof(double) * c->p, cudaMemcpyDeviceToDevice,
                             c->stream));
  int r = centre_kernels(c);
  if (!r) r = refresh_cache(c);
  return r;
}

int smc_reweight(smc_ctx *c, double *a_next, double *log_z_inc, double *ess) {
  if (!c) return SMC_ERR_ARG;
  c->stage += 1;
  if (!c->stage_dev) c->dev_stage_synced = false;
  c->moves_in_stage = 0;
  int nl = 0;
  int e;
  if (c->cv_centre == 2 && !c->full_data) {  // centre at the current cloud, then reweight
    ProfScope ps(c, 4);
    LAUNCH(c,
           weighted_moments(c->is_f64, c->N, c->p, c->W, c->theta, c->part, c->mean_d,
                            c->Sigma_raw, c->stream),
           4);
    const int r0 = recentre(c);
    if (r0) return r0;
  }
  {
    ProfScope ps(c, 3);
    e = reweight(c->N, c->ell, c->sig2, c->logW, c->W, c->tau, c->K, c->rounds, c->grid_points,
                 c->grid_decades, c->st, c->part, &nl, c->stream, !c->batch_member);
  }
  c->launches += nl;
  if (e) return fail(c, SMC_ERR_CUDA, std::string("reweight: ") + cudaGetErrorString((cudaError_t)e));
  int r;
  {
    ProfScope ps(c, 4);
    LAUNCH(c,
           weighted_moments(c->is_f64, c->N, c->p, c->W, c->theta, c->part, c->mean_d,
                            c->Sigma_raw, c->stream),
           4);
    r = set_mass(c);
  }
  if (r) return r;
  if (c->cv_centre == 1 && !c->full_data) {  // Algorithm 2 (d): centre at the reweighted mean
    ProfScope ps(c, 4);
    if ((r = recentre(c))) return r;
  }
  if (a_next || log_z_inc || ess) {
    DevState h;
    if ((r = sync_state(c, &h))) return r;
    if (a_next) *a_next = h.a;
    if (log_z_inc) *log_z_inc = h.log_z_inc;
    if (ess) *ess = h.ess;
    return check_err_bits(c, h);
  }
  return SMC_OK;
}

int smc_resample(smc_ctx *c, int32_t *ancestors) {
  if (!c) return SMC_ERR_ARG;
  ProfScope ps(c, 5);
  LAUNCH(c,
         resample(c->is_f64, c->N, c->p, c->m, c->G, c->seed, c->stage, c->stage_dev,
                  c->multinomial, c->W,
                  c->cum, c->anc,
                  c->theta, c->theta_alt, c->u, c->u_alt, c->ell, c->ell_alt, c->sig2,
                  c->sig2_alt, c->blk, c->blk_alt, c->logW, c->W, c->st, c->stream),
         3);
  std::swap(c->theta, c->theta_alt);
  std::swap(c->u, c->u_alt);
  std::swap(c->ell, c->ell_alt);
  std::swap(c->sig2, c->sig2_alt);
  std::swap(c->blk, c->blk_alt);
  c->parity ^= 1;
  if (ancestors)
    CUDA_OK(c, cudaMemcpyAsync(ancestors, c->anc, sizeof(int32_t) * c->N, cudaMemcpyDefault,
                               c->stream));
  return SMC_OK;
}

static int full_moves(smc_ctx *c, int R);

int smc_move(smc_ctx *c, int32_t R, double *acc_u, double *acc_theta) {
  if (!c) return SMC_ERR_ARG;
  if (R < 1) return fail(c, SMC_ERR_ARG, "R must be >= 1");
  if (c->moves_in_stage + R > 256) return fail(c, SMC_ERR_ARG, "at most 256 moves per stage");
  CUDA_OK(c, cudaMemsetAsync(&c->st->acc_u, 0, 2 * sizeof(unsigned long long), c->stream));
  if (c->full_data) {
    int r = full_moves(c, R);
    if (r) return r;
  }
  for (int r = 0; r < (c->full_data ? 0 : R); ++r) {
    EstArgs a = base_args(c);
    a.B = c->shard_count > 0 ? c->shard_count : c->N;
    a.i0 = c->shard_count > 0 ? c->shard_base : 0;
    a.theta = c->theta;
    a.theta_out = c->theta;
    a.u = c->u;
    a.u_mut = c->u;
    a.ell = c->ell;
    a.sig2 = c->sig2;
    a.blk = c->blk;
    a.blk_prop = c->blk_prop;
    a.move = c->moves_in_stage + r;
    a.stage_dev = c->stage_dev;
    LAUNCH(c, est_launch(c, 1, a), 0);
    LAUNCH(c, hmc_launch(c, a), 0);
  }
  c->moves_in_stage += R;
  // a shard leaves the step size to smc_finish_moves (it needs every shard's accept counts)
  if (c->shard_count == 0) LAUNCH(c, eps_update(c->N, R, c->st, c->stream, c->rw ? 0.234 : 0.65), 1);
  if (acc_u || acc_theta) {
    DevState h;
    int r = sync_state(c, &h);
    if (r) return r;
    const double moved = (double)(c->shard_count > 0 ? c->shard_count : c->N) * R;
    if (acc_u) *acc_u = (double)h.acc_u / moved;
    if (acc_theta) *acc_theta = (double)h.acc_theta / moved;
    return check_err_bits(c, h);
  }
  return SMC_OK;
}

// Moves until the particles have decorrelated from the cloud they started the stage's moves from
// (the number of moves R tuned as in Buchholz et al., cited in Sec. 3.4): after each move the
// componentwise correlations rho_c between the starting and the current cloud are formed, and the
// moves stop once the quantile-q order statistic of rho_1..rho_p (the ceil(q p)-th smallest) is at
// most rho_max, or after R_max moves. The step-size rule then sees the acceptance over the moves
// made. Reads the correlations on the host after every move.
int smc_move_adaptive(smc_ctx *c, int32_t R_max, double rho_max, double quantile,
                      int32_t *R_used, double *acc_u, double *acc_theta) {
  if (!c) return SMC_ERR_ARG;
  if (R_max < 1 || c->moves_in_stage + R_max > 256)
    return fail(c, SMC_ERR_ARG, "R_max must be >= 1, at most 256 moves per stage");
  if (!(rho_max >= -1.0 && rho_max <= 1.0) || !(quantile > 0.0 && quantile <= 1.0))
    return fail(c, SMC_ERR_ARG, "rho_max must be in [-1, 1] and quantile in (0, 1]");
  if (c->capturing) return fail(c, SMC_ERR_ARG, "adaptive moves cannot be graph-captured");
  if (c->shard_count > 0) return fail(c, SMC_ERR_STATE, "adaptive moves are not sharded");
  const int N = c->N, p = c->p;
  const size_t tbytes = (size_t)N * p * (c->is_f64 ? sizeof(double) : sizeof(float));
  if (!c->theta0) {
    ALLOC(c, c->theta0, tbytes);
    ALLOC(c, c->rho_d, sizeof(double) * p);
  }
  CUDA_OK(c, cudaMemsetAsync(&c->st->acc_u, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_OK(c, cudaMemcpyAsync(c->theta0, c->theta, tbytes, cudaMemcpyDeviceToDevice, c->stream));
  int kq = (int)ceil(quantile * p) - 1;
  kq = kq < 0 ? 0 : (kq >= p ? p - 1 : kq);
  std::vector<double> rho(p);
  int R = 0;
  while (R < R_max) {
    if (c->full_data) {
      int r = full_moves(c, 1);
      if (r) return r;
    } else {
      EstArgs a = base_args(c);
      a.B = N;
      a.theta = c->theta;
      a.theta_out = c->theta;
      a.u = c->u;
      a.u_mut = c->u;
      a.ell = c->ell;
      a.sig2 = c->sig2;
      a.blk = c->blk;
      a.blk_prop = c->blk_prop;
      a.move = c->moves_in_stage;
      a.stage_dev = c->stage_dev;
      LAUNCH(c, est_launch(c, 1, a), 0);
      LAUNCH(c, hmc_launch(c, a), 0);
    }
    c->moves_in_stage += 1;
    R += 1;
    LAUNCH(c, autocorr(c->is_f64, N, p, c->theta0, c->theta, c->rho_d, c->stream), 1);
    CUDA_OK(c, cudaMemcpyAsync(rho.data(), c->rho_d, sizeof(double) * p, cudaMemcpyDeviceToHost,
                               c->stream));
    CUDA_OK(c, cudaStreamSynchronize(c->stream));
    std::vector<double> sorted(rho);
    std::sort(sorted.begin(), sorted.end());
    if (sorted[kq] <= rho_max) break;
  }
  LAUNCH(c, eps_update(N, R, c->st, c->stream, c->rw ? 0.234 : 0.65), 1);
  if (R_used) *R_used = R;
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  if (acc_u) *acc_u = (double)h.acc_u / ((double)N * R);
  if (acc_theta) *acc_theta = (double)h.acc_theta / ((double)N * R);
  return check_err_bits(c, h);
}

// The host-side effects of one stage, mirrored on a graph replay: stage counters, the resampling
// buffer swap, the launch count.
static void mirror_stage(smc_ctx *c, int R, int q) {
  c->stage += 1;
  c->moves_in_stage = R;
  std::swap(c->theta, c->theta_alt);
  std::swap(c->u, c->u_alt);
  std::swap(c->ell, c->ell_alt);
  std::swap(c->sig2, c->sig2_alt);
  std::swap(c->blk, c->blk_alt);
  c->parity ^= 1;
  c->launches += c->g_launches[q];
}

static int stage_body(smc_ctx *c, int R) {
  int r = smc_reweight(c, nullptr, nullptr, nullptr);
  if (!r) r = smc_resample(c, nullptr);
  if (!r) r = smc_move(c, R, nullptr, nullptr);
  return r;
}

int smc_stage(smc_ctx *c, int32_t R, int32_t use_graph) {
  if (!c) return SMC_ERR_ARG;
  if (R < 1 || R > 256) return fail(c, SMC_ERR_ARG, "R must be in [1, 256]");
  if (!use_graph) return stage_body(c, R);
  if (!c->dev_stage_synced) {
    LAUNCH(c, stage_set(c->st, c->stage, c->stream), 1);
    c->dev_stage_synced = true;
  }
  const int q = c->parity;
  if (c->gexec[q] && c->g_R[q] == R) {
    CUDA_OK(c, cudaGraphLaunch(c->gexec[q], c->stream));
    mirror_stage(c, R, q);
    return SMC_OK;
  }
  if (c->gexec[q]) {
    cudaGraphExecDestroy(c->gexec[q]);
    c->gexec[q] = nullptr;
  }
  // Capture on a private stream (the legacy default stream cannot be captured). Capturing runs the
  // stage's host code, which advances the host-side state as if the stage had run; the graph is
  // launched right after, on the context's stream, so device and host agree again.
  cudaStream_t cap;
  CUDA_OK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaStream_t orig = c->stream;
  const int64_t l0 = c->launches;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) {
    cudaStreamDestroy(cap);
    return fail(c, SMC_ERR_CUDA, std::string("stage capture: ") + cudaGetErrorString(e));
  }
  c->stream = cap;
  c->capturing = true;
  c->stage_dev = 1;
  int r = stage_advance(c->st, cap);
  c->launches += 1;
  if (!r) r = stage_body(c, R);
  cudaGraph_t g = nullptr;
  const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  c->stream = orig;
  c->capturing = false;
  c->stage_dev = 0;
  cudaStreamDestroy(cap);
  if (r || e2 != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    c->dev_stage_synced = false;
    if (r) return r;
    return fail(c, SMC_ERR_CUDA, std::string("stage capture: ") + cudaGetErrorString(e2));
  }
  e = cudaGraphInstantiate(&c->gexec[q], g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    c->gexec[q] = nullptr;
    return fail(c, SMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
  }
  c->g_R[q] = R;
  c->g_launches[q] = c->launches - l0;
  CUDA_OK(c, cudaGraphLaunch(c->gexec[q], c->stream));
  return SMC_OK;
}

static int estimate_impl(smc_ctx *c, int32_t B, const void *theta, const int32_t *u, double a,
                         void *grad, double *ell, double *sigma2) {
  if (!c) return SMC_ERR_ARG;
  if (B < 0 || (B > 0 && (!theta || !u))) return fail(c, SMC_ERR_ARG, "bad batch arguments");
  EstArgs ea = base_args(c);
  ea.B = B;
  ea.theta = theta;
  ea.u = u;
  ea.ell = ell;
  ea.sig2 = sigma2;
  ea.grad = grad;
  ea.a_host = a;
  LAUNCH(c, est_launch(c, 0, ea), 0);
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  return check_err_bits(c, h);
}

int loglik_est(smc_ctx *c, int32_t B, const void *theta, const int32_t *u, double *ell,
               double *sigma2) {
  return estimate_impl(c, B, theta, u, 0.0, nullptr, ell, sigma2);
}

int loglik_grad(smc_ctx *c, int32_t B, const void *theta, const int32_t *u, double a, void *grad,
                double *ell, double *sigma2) {
  if (!grad) return fail(c, SMC_ERR_ARG, "grad is NULL");
  return estimate_impl(c, B, theta, u, a, grad, ell, sigma2);
}

int loglik_fwd(smc_ctx *c, int32_t B, const void *theta, const int32_t *u, double *ell,
               double *sigma2, void *d_save, void *r_save) {
  if (!c) return SMC_ERR_ARG;
  if (B < 0 || (B > 0 && (!theta || !u || !ell || !sigma2 || !d_save || !r_save)))
    return fail(c, SMC_ERR_ARG, "bad loglik_fwd arguments");
  EstArgs ea = base_args(c);
  ea.B = B;
  ea.theta = theta;
  ea.u = u;
  ea.ell = ell;
  ea.sig2 = sigma2;
  ea.dsave = d_save;
  ea.rsave = r_save;
  LAUNCH(c, est_launch(c, 3, ea), 0);
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  return check_err_bits(c, h);
}

int loglik_bwd(smc_ctx *c, int32_t B, const void *theta, const int32_t *u, const void *d_save,
               const void *r_save, const double *g_ell, const double *g_sig2, void *grad) {
  if (!c) return SMC_ERR_ARG;
  if (B < 0 || (B > 0 && (!theta || !u || !d_save || !r_save || !g_ell || !g_sig2 || !grad)))
    return fail(c, SMC_ERR_ARG, "bad loglik_bwd arguments");
  EstArgs ea = base_args(c);
  ea.B = B;
  ea.theta = theta;
  ea.u = u;
  ea.dsave = const_cast<void *>(d_save);
  ea.rsave = const_cast<void *>(r_save);
  ea.g_ell = g_ell;
  ea.g_sig2 = g_sig2;
  ea.grad = grad;
  LAUNCH(c, est_launch(c, 4, ea), 0);
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  return check_err_bits(c, h);
}

int loglik_full(smc_ctx *c, int32_t B, const void *theta, double a, double *ell, void *grad) {
  if (!c) return SMC_ERR_ARG;
  if (B < 0 || (B > 0 && !theta) || (!ell && !grad))
    return fail(c, SMC_ERR_ARG, "bad loglik_full arguments");
  int r = full_prepare(c, B);
  if (r) return r;
  if (B == 0) return SMC_OK;
  if ((r = full_eval(c, B, theta, a, nullptr, ell, grad))) return r;
  return full_check_flag(c);
}

// R HMC moves of the full-data comparison SMC: per move the momentum and H0, then the leapfrog
// loop (L + 1 full-data evaluations with kicks and drifts between them; replayed as one CUDA
// graph after its first capture), then the Metropolis-Hastings step with the exact l at the end
// point. Inside a stage capture (smc_stage) the loop is captured inline instead.
static int full_leapfrog(smc_ctx *c) {
  const int N = c->N, p = c->p;
  const double *adev = &c->st->a;
  int r = full_eval(c, N, c->fm_thp, 0.0, adev, nullptr, c->fm_g);
  if (r) return r;
  for (int l = 0; l < c->L; ++l) {
    LAUNCH(c, full_move_kick(N, p, c->fm_thp, c->fm_rho, c->fm_g, c->Sigma_ct, c->fm_eps, 1,
                             c->stream),
           1);
    if ((r = full_eval(c, N, c->fm_thp, 0.0, adev, c->fm_ell, c->fm_g))) return r;
    LAUNCH(c, full_move_kick(N, p, c->fm_thp, c->fm_rho, c->fm_g, c->Sigma_ct, c->fm_eps, 0,
                             c->stream),
           1);
  }
  return SMC_OK;
}

static int full_moves(smc_ctx *c, int R) {
  const int N = c->N, p = c->p;
  for (int q = 0; q < R; ++q) {
    const int move = c->moves_in_stage + q;
    LAUNCH(c,
           full_move_begin(N, p, c->theta, c->fm_thp, c->fm_rho, c->Linv_ct, c->Sigma_ct, c->mu_ct,
                           c->ivar_ct, c->ell, c->seed, c->stage, c->stage_dev, move, c->st,
                           c->fm_h0, c->eps_jitter, c->fm_eps, c->stream),
           1);
    if (c->capturing) {
      int r = full_leapfrog(c);
      if (r) return r;
    } else {
      if (!c->fm_graph) {  // capture the loop once (its buffers and sizes never change)
        cudaStream_t cap;
        CUDA_OK(c, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
        cudaStream_t orig = c->stream;
        cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) {
          cudaStreamDestroy(cap);
          return fail(c, SMC_ERR_CUDA, std::string("leapfrog capture: ") + cudaGetErrorString(e));
        }
        c->stream = cap;
        c->capturing = true;
        const int64_t l0 = c->launches;
        int r = full_leapfrog(c);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(cap, &g);
        c->stream = orig;
        c->capturing = false;
        cudaStreamDestroy(cap);
        c->fm_launches = c->launches - l0;
        c->launches = l0;
        if (r || e != cudaSuccess || !g) {
          if (g) cudaGraphDestroy(g);
          if (r) return r;
          return fail(c, SMC_ERR_CUDA, std::string("leapfrog capture: ") + cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&c->fm_graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          c->fm_graph = nullptr;
          return fail(c, SMC_ERR_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(e));
        }
      }
      CUDA_OK(c, cudaGraphLaunch(c->fm_graph, c->stream));
      c->launches += c->fm_launches;
    }
    LAUNCH(c,
           full_move_accept(N, p, c->theta, c->fm_thp, c->fm_rho, c->Sigma_ct, c->mu_ct, c->ivar_ct,
                            c->ell, c->fm_ell, c->fm_h0, c->seed, c->stage, c->stage_dev, move,
                            c->st, c->stream),
           1);
  }
  return SMC_OK;
}

int smc_get_particles(smc_ctx *c, void *theta, int32_t *u, double *W) {
  if (!c) return SMC_ERR_ARG;
  if (theta)
    CUDA_OK(c, cudaMemcpyAsync(theta, c->theta, ct_size(c) * c->N * c->p, cudaMemcpyDefault,
                               c->stream));
  if (u)
    CUDA_OK(c, cudaMemcpyAsync(u, c->u, sizeof(int32_t) * c->N * c->m, cudaMemcpyDefault,
                               c->stream));
  if (W) CUDA_OK(c, cudaMemcpyAsync(W, c->W, sizeof(double) * c->N, cudaMemcpyDefault, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_set_particles(smc_ctx *c, const void *theta, const int32_t *u, const double *W) {
  if (!c) return SMC_ERR_ARG;
  if (theta)
    CUDA_OK(c, cudaMemcpyAsync(c->theta, theta, ct_size(c) * c->N * c->p, cudaMemcpyDefault,
                               c->stream));
  if (u)
    CUDA_OK(c, cudaMemcpyAsync(c->u, u, sizeof(int32_t) * c->N * c->m, cudaMemcpyDefault,
                               c->stream));
  double *Wd = nullptr;
  if (W) {
    Wd = c->ell_alt;  // staging buffer of N doubles
    CUDA_OK(c, cudaMemcpyAsync(Wd, W, sizeof(double) * c->N, cudaMemcpyDefault, c->stream));
  }
  LAUNCH(c, weights_from(c->N, Wd, c->logW, c->W, c->stream), 1);
  int r = refresh_cache(c);
  if (r) return r;
  DevState h;
  if ((r = sync_state(c, &h))) return r;
  return check_err_bits(c, h);
}

int smc_get_cache(smc_ctx *c, double *ell, double *sigma2, double *blocks) {
  if (!c) return SMC_ERR_ARG;
  if (ell)
    CUDA_OK(c, cudaMemcpyAsync(ell, c->ell, sizeof(double) * c->N, cudaMemcpyDefault, c->stream));
  if (sigma2)
    CUDA_OK(c, cudaMemcpyAsync(sigma2, c->sig2, sizeof(double) * c->N, cudaMemcpyDefault,
                               c->stream));
  if (blocks)
    CUDA_OK(c, cudaMemcpyAsync(blocks, c->blk, sizeof(double) * c->N * c->G * 2,
                               cudaMemcpyDefault, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_get_centre(smc_ctx *c, double *theta_bar, double *A, double *B, double *C) {
  if (!c) return SMC_ERR_ARG;
  const int p = c->p;
  if (theta_bar)
    CUDA_OK(c, cudaMemcpyAsync(theta_bar, c->tb_d, sizeof(double) * p, cudaMemcpyDeviceToHost,
                               c->stream));
  if (A) CUDA_OK(c, cudaMemcpyAsync(A, c->A_d, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (B)
    CUDA_OK(c, cudaMemcpyAsync(B, c->B_d, sizeof(double) * p, cudaMemcpyDeviceToHost, c->stream));
  if (C)
    CUDA_OK(c, cudaMemcpyAsync(C, c->C_d, sizeof(double) * p * p, cudaMemcpyDeviceToHost,
                               c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_cv_moments(smc_ctx *c, const double *theta, double *A, double *B, double *C) {
  if (!c || !theta) return SMC_ERR_ARG;
  const int p = c->p;
  double *th = c->scratch_d, *A1 = th + p, *B1 = A1 + 1, *C1 = B1 + p;
  CUDA_OK(c, cudaMemcpyAsync(th, theta, sizeof(double) * p, cudaMemcpyHostToDevice, c->stream));
  int r = moments_at(c, th, A1, B1, C1);
  if (r) return r;
  if (A) CUDA_OK(c, cudaMemcpyAsync(A, A1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  if (B) CUDA_OK(c, cudaMemcpyAsync(B, B1, sizeof(double) * p, cudaMemcpyDeviceToHost, c->stream));
  if (C)
    CUDA_OK(c, cudaMemcpyAsync(C, C1, sizeof(double) * p * p, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_get_mass(smc_ctx *c, double *Sigma, double *chol) {
  if (!c) return SMC_ERR_ARG;
  const size_t b = sizeof(double) * c->p * c->p;
  if (Sigma) CUDA_OK(c, cudaMemcpyAsync(Sigma, c->Sigma_d, b, cudaMemcpyDeviceToHost, c->stream));
  if (chol) CUDA_OK(c, cudaMemcpyAsync(chol, c->chol_d, b, cudaMemcpyDeviceToHost, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_get_status(smc_ctx *c, double *a, double *log_z, int32_t *stage, double *eps) {
  if (!c) return SMC_ERR_ARG;
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  if (a) *a = h.a;
  if (log_z) *log_z = h.log_z;
  if (stage) *stage = c->stage;
  if (eps) *eps = h.eps;
  return SMC_OK;
}

int smc_set_scalars(smc_ctx *c, int32_t stage, double a, double eps, double log_z) {
  if (!c) return SMC_ERR_ARG;
  if (stage < 0 || !(a >= 0 && a <= 1) || !(eps > 0)) return fail(c, SMC_ERR_ARG, "bad scalars");
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  h.a = a;
  h.eps = eps;
  h.log_z = log_z;
  CUDA_OK(c, cudaMemcpyAsync(c->st, &h, sizeof(DevState), cudaMemcpyHostToDevice, c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  c->stage = stage;
  c->moves_in_stage = 0;
  c->dev_stage_synced = false;
  return SMC_OK;
}

int smc_autotune(smc_ctx *c, int32_t *tile, int32_t *hmc_kernel) {
  if (!c) return SMC_ERR_ARG;
  Tile tl[32];
  const int nt = est_tiles(c, tl, 32);
  cudaEvent_t e0, e1;
  CUDA_OK(c, cudaEventCreate(&e0));
  CUDA_OK(c, cudaEventCreate(&e1));
  auto time_it = [&](auto &&launch, int reps, float *out_ms) -> int {
    float total = 0.f;
    for (int rep = 0; rep < reps + 1; ++rep) {
      CUDA_OK(c, cudaEventRecord(e0, c->stream));
      LAUNCH(c, launch(), 0);
      CUDA_OK(c, cudaEventRecord(e1, c->stream));
      CUDA_OK(c, cudaEventSynchronize(e1));
      float ms = 0.f;
      CUDA_OK(c, cudaEventElapsedTime(&ms, e0, e1));
      if (rep) total += ms;  // the first launch is a warm-up
    }
    *out_ms = total;
    return SMC_OK;
  };
  // 1. estimator tile (plain estimator with gradient on the context's particles)
  int best = c->tile;
  float best_ms = 1e30f;
  for (int t = 0; t < nt; ++t) {
    if (tl[t].T * tl[t].CPL < c->Sx) continue;
    c->tile = t;
    EstArgs a = base_args(c);
    a.B = c->N;
    a.theta = c->theta;
    a.u = c->u;
    a.grad = c->grad_scratch;
    a.a_host = 1.0;
    float ms = 0.f;
    int r = time_it([&]() { return est_launch(c, 0, a); }, 3, &ms);
    if (r) return r;
    if (ms < best_ms) {
      best_ms = ms;
      best = t;
    }
  }
  c->tile = best;
  // 2. HMC trajectory kernel, on scratch copies (theta_alt, ell_alt, sig2_alt, blk_alt)
  const size_t cts = ct_size(c);
  CUDA_OK(c, cudaMemcpyAsync(c->theta_alt, c->theta, cts * c->N * c->p, cudaMemcpyDeviceToDevice,
                             c->stream));
  EstArgs a = base_args(c);
  a.B = c->N;
  a.theta = c->theta_alt;
  a.theta_out = c->theta_alt;
  a.u = c->u;
  a.ell = c->ell_alt;
  a.sig2 = c->sig2_alt;
  a.blk = c->blk_alt;
  a.blk_prop = c->blk_prop;
  a.move = 255;
  // The default kernel is timed first and stays unless another is faster by more than 3%: the
  // candidates are timed on the initial particles only, where near-equal tiles trade places by
  // noise, while the default is the one chosen for the whole run's range of stages.
  const int keep_res = c->res_tile;
  const int def_res = c->rw ? -1 : default_res_tile(c);
  int best_res = def_res;
  float best_hmc = 1e30f;
  Tile tr[32];
  const int nr = res_tiles(c, tr, 32);
  for (int k = -2; k < nr; ++k) {
    const int t = k == -2 ? def_res : k;  // the default first, then every candidate
    if (k >= -1 && t == def_res) continue;
    if (t >= 0 && res_launch(c, t, a, true) != 0) continue;
    c->res_tile = t;
    float ms = 0.f;
    int r = time_it([&]() { return hmc_launch(c, a); }, 2, &ms);
    if (r) {
      c->res_tile = keep_res;
      return r;
    }
    if (k == -2 ? true : ms < 0.97f * best_hmc) {
      best_hmc = ms;
      best_res = t;
    }
  }
  c->res_tile = best_res;
  drop_graphs(c);  // captured stages used the previous kernels
  CUDA_OK(c, cudaMemsetAsync(&c->st->acc_u, 0, 2 * sizeof(unsigned long long), c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tile) *tile = best + 1;
  if (hmc_kernel) *hmc_kernel = best_res < 0 ? 1 : best_res + 2;
  return SMC_OK;
}

int64_t smc_launch_count(const smc_ctx *c) { return c ? c->launches : 0; }

int smc_profile_enable(smc_ctx *c, int32_t on) {
  if (!c) return SMC_ERR_ARG;
  c->prof_on = on != 0;
  return SMC_OK;
}

int smc_profile_read(smc_ctx *c, int32_t group, int64_t *launches, double *total_ms) {
  if (!c || group < 0 || group > 5) return SMC_ERR_ARG;
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  double tot = 0.0;
  for (auto &pr : c->prof[group]) {
    float ms = 0.f;
    CUDA_OK(c, cudaEventElapsedTime(&ms, pr.first, pr.second));
    tot += ms;
    c->ev_pool.push_back(pr.first);
    c->ev_pool.push_back(pr.second);
  }
  if (launches) *launches = (int64_t)c->prof[group].size();
  if (total_ms) *total_ms = tot;
  c->prof[group].clear();
  return SMC_OK;
}

// ------------------------------------------------------------------------------------------------
// Particle shards: slices of one posterior's particles on several processes (see subsmc.h).
// ------------------------------------------------------------------------------------------------
namespace {
// rows[k] = u[idx[k]] (dir 0) or u[idx[k]] = rows[k] (dir 1); one warp per listed particle.
__global__ void k_shard_rows(int count, int N, int m, const int32_t *idx, int32_t *u,
                             int32_t *rows, int dir, DevState *st) {
  const int lane = threadIdx.x & 31;
  const int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k >= count) return;
  const int i = idx[k];
  if (i < 0 || i >= N) {
    if (lane == 0) atomicOr(&st->err, kErrIndex);
    return;
  }
  int32_t *ur = u + (int64_t)i * m, *rr = rows + (int64_t)k * m;
  for (int j = lane; j < m; j += 32) {
    if (dir == 0)
      rr[j] = ur[j];
    else
      ur[j] = rr[j];
  }
}
int shard_rows(smc_ctx *c, int32_t count, const int32_t *idx, int32_t *rows, int32_t *u, int dir) {
  if (count < 0 || (count > 0 && (!idx || !rows)))
    return fail(c, SMC_ERR_ARG, "shard rows: bad arguments");
  if (count == 0) return SMC_OK;
  const int wpb = 8;
  k_shard_rows<<<(count + wpb - 1) / wpb, wpb * 32, 0, c->stream>>>(count, c->N, c->m, idx, u,
                                                                    rows, dir, c->st);
  c->launches += 1;
  CUDA_OK(c, cudaGetLastError());
  return SMC_OK;
}
}  // namespace

extern "C" {

int smc_shard_export(smc_ctx *c, void *theta, double *ell, double *sigma2, double *blocks) {
  if (!c) return SMC_ERR_ARG;
  if (c->shard_count == 0) return fail(c, SMC_ERR_STATE, "the context has no shard");
  const size_t b = (size_t)c->shard_base, n = (size_t)c->shard_count, cts = ct_size(c);
  const size_t G2 = (size_t)c->G * 2;
  if (theta)
    CUDA_OK(c, cudaMemcpyAsync(theta, (char *)c->theta + b * c->p * cts, n * c->p * cts,
                               cudaMemcpyDefault, c->stream));
  if (ell)
    CUDA_OK(c, cudaMemcpyAsync(ell, c->ell + b, n * sizeof(double), cudaMemcpyDefault, c->stream));
  if (sigma2)
    CUDA_OK(c, cudaMemcpyAsync(sigma2, c->sig2 + b, n * sizeof(double), cudaMemcpyDefault,
                               c->stream));
  if (blocks)
    CUDA_OK(c, cudaMemcpyAsync(blocks, c->blk + b * G2, n * G2 * sizeof(double), cudaMemcpyDefault,
                               c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_shard_import(smc_ctx *c, const void *theta, const double *ell, const double *sigma2,
                     const double *blocks) {
  if (!c) return SMC_ERR_ARG;
  const size_t N = (size_t)c->N, G2 = (size_t)c->G * 2;
  if (theta)
    CUDA_OK(c, cudaMemcpyAsync(c->theta, theta, N * c->p * ct_size(c), cudaMemcpyDefault,
                               c->stream));
  if (ell) CUDA_OK(c, cudaMemcpyAsync(c->ell, ell, N * sizeof(double), cudaMemcpyDefault, c->stream));
  if (sigma2)
    CUDA_OK(c, cudaMemcpyAsync(c->sig2, sigma2, N * sizeof(double), cudaMemcpyDefault, c->stream));
  if (blocks)
    CUDA_OK(c, cudaMemcpyAsync(c->blk, blocks, N * G2 * sizeof(double), cudaMemcpyDefault,
                               c->stream));
  CUDA_OK(c, cudaStreamSynchronize(c->stream));
  return SMC_OK;
}

int smc_shard_gather_u(smc_ctx *c, int32_t count, const int32_t *idx, int32_t *rows,
                       int32_t before_resample) {
  if (!c) return SMC_ERR_ARG;
  return shard_rows(c, count, idx, rows, before_resample ? c->u_alt : c->u, 0);
}

int smc_shard_scatter_u(smc_ctx *c, int32_t count, const int32_t *idx, const int32_t *rows) {
  if (!c) return SMC_ERR_ARG;
  return shard_rows(c, count, idx, const_cast<int32_t *>(rows), c->u, 1);
}

int smc_move_accepts(smc_ctx *c, uint64_t *acc_u, uint64_t *acc_theta) {
  if (!c) return SMC_ERR_ARG;
  DevState h;
  int r = sync_state(c, &h);
  if (r) return r;
  if (acc_u) *acc_u = h.acc_u;
  if (acc_theta) *acc_theta = h.acc_theta;
  return check_err_bits(c, h);
}

int smc_finish_moves(smc_ctx *c, int32_t R, uint64_t acc_u, uint64_t acc_theta) {
  if (!c) return SMC_ERR_ARG;
  if (R < 1) return fail(c, SMC_ERR_ARG, "R must be >= 1");
  unsigned long long v[2] = {acc_u, acc_theta};
  CUDA_OK(c, cudaMemcpyAsync(&c->st->acc_u, v, sizeof(v), cudaMemcpyHostToDevice, c->stream));
  LAUNCH(c, eps_update(c->N, R, c->st, c->stream, c->rw ? 0.234 : 0.65), 1);
  CUDA_OK(c, cudaStreamSynchronize(c->stream));  // v lives on this stack frame
  return SMC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------------------------------
// Batches of independent posteriors (many problems of uneven n and p stepped together): one context
// per problem, and per move one u-update launch and one HMC launch over all particles of all
// problems (the kernels find each particle's problem from the prefix offsets).
// ------------------------------------------------------------------------------------------------
// A group of problems whose trajectories run in one launch: a resident tile (tile >= 0, the
// subsample kept in shared memory; the plan sized by the group's largest p, m and G) or the
// streamed kernel (tile = -1). The group's problems are order[start .. start + count).
struct BatchGroup {
  int tile, start, count, total, pmax, mmax, Gmax;
};

struct smc_batch {
  int P = 0, tile = 0, total = 0, wstride = 0, Rcap = 0;
  std::vector<smc_ctx *> ctx;
  cudaStream_t stream = nullptr;
  int *offsets_d = nullptr;   // [P] first particle of each problem (problem order)
  int *goff_d = nullptr;      // [P] first particle of each problem within its group (sorted order)
  std::vector<int> order;     // problems sorted by group
  std::vector<int> group_of;  // per problem: its group
  std::vector<BatchGroup> groups;
  EstArgs *args_d = nullptr;  // [Rcap] x [2 P]: per move the problems' arguments in problem order,
                              // then in the sorted order of the groups
  std::vector<EstArgs> args_h;
  cudaGraphExec_t gexec[2] = {nullptr, nullptr};
  EstArgs *gargs[2] = {nullptr, nullptr};  // the argument arrays each graph reads
  int gR[2] = {0, 0};
  int64_t glaunches[2] = {0, 0};  // kernel launches inside each graph
  int64_t launches = 0;
  // side streams for the per-problem stage steps (reweighting, moments, resampling): problem q
  // runs on side[q % side.size()], forked from and joined back to the batch stream by events
  std::vector<cudaStream_t> side;
  std::vector<cudaEvent_t> ev_side;
  cudaEvent_t ev_fork = nullptr;
  // batched stage steps (every problem with a fixed centre): the problems' stage arguments per
  // buffer parity and the block offsets of each launch kind
  bool stage_kernels = false;
  StageArgs *sargs_d[2] = {nullptr, nullptr};
  int *soff_d = nullptr;
  StageBatch sb{};
  std::string err;
};

static int bfail(smc_batch *b, int code, const std::string &msg) {
  if (b) b->err = msg;
  return code;
}

// Arguments of move `move` for problem context c; swapped: use the buffers the next resampling
// will make current (for graphs built before the stage's host code runs).
static EstArgs batch_move_args(smc_ctx *c, int move, bool swapped, int stage_dev) {
  EstArgs a = base_args(c);
  a.B = c->N;
  a.theta = a.theta_out = swapped ? c->theta_alt : c->theta;
  a.u = a.u_mut = swapped ? c->u_alt : c->u;
  a.ell = swapped ? c->ell_alt : c->ell;
  a.sig2 = swapped ? c->sig2_alt : c->sig2;
  a.blk = swapped ? c->blk_alt : c->blk;
  a.blk_prop = c->blk_prop;
  a.move = move;
  a.stage_dev = stage_dev;
  return a;
}

static int batch_upload(smc_batch *b, int R, bool swapped, int stage_dev) {
  const size_t P2 = 2 * (size_t)b->P;
  if (R > b->Rcap) {
    if (b->args_d) cudaFree(b->args_d);
    b->args_d = nullptr;
    if (cudaMalloc(&b->args_d, sizeof(EstArgs) * (size_t)R * P2) != cudaSuccess)
      return bfail(b, SMC_ERR_OOM, "batch argument array");
    b->Rcap = R;
  }
  b->args_h.resize((size_t)R * P2);
  for (int r = 0; r < R; ++r)
    for (int q = 0; q < b->P; ++q)
      b->args_h[(size_t)r * P2 + q] =
          batch_move_args(b->ctx[q], swapped ? r : b->ctx[q]->moves_in_stage + r, swapped,
                          stage_dev);
  for (int r = 0; r < R; ++r)
    for (int k = 0; k < b->P; ++k)
      b->args_h[(size_t)r * P2 + b->P + k] = b->args_h[(size_t)r * P2 + b->order[k]];
  // synchronous with respect to the host (pageable source), before any capture begins
  if (cudaMemcpyAsync(b->args_d, b->args_h.data(), sizeof(EstArgs) * (size_t)R * P2,
                      cudaMemcpyHostToDevice, b->stream) != cudaSuccess)
    return bfail(b, SMC_ERR_CUDA, "batch argument upload");
  return SMC_OK;
}

// Per move: one u-update launch over all problems (streamed rows), then one trajectory launch
// per group (resident tile, or the streamed kernel for problems no resident tile takes). The
// groups touch disjoint problems, so their launches run side by side on the side streams (forked
// from and joined back to the batch stream: one group's tail overlaps the others' work).
static int batch_moves(smc_batch *b, int R) {
  const size_t P2 = 2 * (size_t)b->P;
  const int sms = b->ctx[0]->sms;
  const int ng = (int)b->groups.size();
  const int nfork = ng > 1 ? std::min(ng, (int)b->side.size()) : 0;
  for (int r = 0; r < R; ++r) {
    BatchArgs ba;
    ba.probs = b->args_d + (size_t)r * P2;
    ba.offsets = b->offsets_d;
    ba.nprob = b->P;
    ba.total = b->total;
    ba.wstride = b->wstride;
    int e = est_launch_batch_bf16(1, b->tile, ba, b->stream);
    b->launches += 1;
    if (!e && nfork > 0) {
      e = (int)cudaEventRecord(b->ev_fork, b->stream);
      for (int k = 0; k < nfork && !e; ++k) e = (int)cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
    }
    for (int g = 0; g < ng && !e; ++g) {
      const BatchGroup &gr = b->groups[g];
      cudaStream_t st = nfork > 0 ? b->side[g % nfork] : b->stream;
      BatchArgs bg;
      bg.probs = b->args_d + (size_t)r * P2 + b->P + gr.start;
      bg.offsets = b->goff_d + gr.start;
      bg.nprob = gr.count;
      bg.total = gr.total;
      bg.wstride = b->wstride;
      e = gr.tile >= 0 ? res_launch_batch_bf16(gr.tile, bg, gr.pmax, gr.mmax, gr.Gmax, st, sms,
                                               false)
                       : est_launch_batch_bf16(2, b->tile, bg, st);
      b->launches += 1;
    }
    for (int k = 0; k < nfork && !e; ++k) {
      e = (int)cudaEventRecord(b->ev_side[k], b->side[k]);
      if (!e) e = (int)cudaStreamWaitEvent(b->stream, b->ev_side[k], 0);
    }
    if (e) return bfail(b, SMC_ERR_CUDA, std::string("batched move: ") +
                                             cudaGetErrorString((cudaError_t)e));
  }
  return SMC_OK;
}

// True when this stage can run the batched stage kernels: every problem has a fixed centre (set
// at init) and all are at the same buffer parity.
static bool batch_stage_kernels(const smc_batch *b) {
  if (!b->stage_kernels) return false;
  for (const smc_ctx *c : b->ctx)
    if (c->parity != b->ctx[0]->parity) return false;
  return true;
}

// The stage of every problem with the batched stage kernels: the temperature search, reweighting,
// moments, mass matrices and resampling of all problems in about 2 rounds + 12 launches, then R
// batched moves and the step sizes. The device stage counters are advanced by the first launch.
static int batch_stage_batched(smc_batch *b, int R, bool args_ready) {
  for (smc_ctx *c : b->ctx) {
    if (!c->dev_stage_synced) {  // outside a capture: a per-problem call left the counter stale
      if (stage_set(c->st, c->stage, b->stream)) return bfail(b, SMC_ERR_CUDA, "stage counter");
      c->dev_stage_synced = true;
    }
  }
  StageBatch sb = b->sb;
  sb.args = b->sargs_d[b->ctx[0]->parity];
  if (stage_batch(sb, b->stream, &b->launches))
    return bfail(b, SMC_ERR_CUDA, "batched stage steps");
  for (smc_ctx *c : b->ctx) {  // the host side of smc_reweight and smc_resample
    c->stage += 1;
    c->moves_in_stage = 0;
    std::swap(c->theta, c->theta_alt);
    std::swap(c->u, c->u_alt);
    std::swap(c->ell, c->ell_alt);
    std::swap(c->sig2, c->sig2_alt);
    std::swap(c->blk, c->blk_alt);
    c->parity ^= 1;
  }
  if (!args_ready) {
    int r = batch_upload(b, R, false, 0);
    if (r) return r;
  }
  int r = batch_moves(b, R);
  if (r) return r;
  for (smc_ctx *c : b->ctx) c->moves_in_stage += R;
  if (eps_update_batch(sb, R, b->stream)) return bfail(b, SMC_ERR_CUDA, "step size");
  b->launches += 1;
  return SMC_OK;
}

// The stage of every problem: reweight and resample per problem, R batched moves, step sizes.
static int batch_stage_body(smc_batch *b, int R, bool args_ready) {
  if (batch_stage_kernels(b)) return batch_stage_batched(b, R, args_ready);
  // the problems' reweighting and resampling are independent: side streams run them side by
  // side (inside a capture they become parallel branches of the graph)
  const int ns = (int)b->side.size();
  if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess)
    return bfail(b, SMC_ERR_CUDA, "stage fork");
  for (int k = 0; k < ns; ++k)
    if (cudaStreamWaitEvent(b->side[k], b->ev_fork, 0) != cudaSuccess)
      return bfail(b, SMC_ERR_CUDA, "stage fork");
  for (int q = 0; q < b->P; ++q) {
    smc_ctx *c = b->ctx[q];
    cudaStream_t own = c->stream;
    c->stream = b->side[q % ns];
    int r = smc_reweight(c, nullptr, nullptr, nullptr);
    if (!r) r = smc_resample(c, nullptr);
    if (!r && cudaMemsetAsync(&c->st->acc_u, 0, 2 * sizeof(unsigned long long), c->stream) !=
                  cudaSuccess)
      r = fail(c, SMC_ERR_CUDA, "accept counters");
    c->stream = own;
    if (r) return bfail(b, r, c->err);
  }
  for (int k = 0; k < ns; ++k) {
    if (cudaEventRecord(b->ev_side[k], b->side[k]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev_side[k], 0) != cudaSuccess)
      return bfail(b, SMC_ERR_CUDA, "stage join");
  }
  if (!args_ready) {
    int r = batch_upload(b, R, false, 0);
    if (r) return r;
  }
  int r = batch_moves(b, R);
  if (r) return r;
  for (smc_ctx *c : b->ctx) {
    c->moves_in_stage += R;
    if (eps_update(c->N, R, c->st, c->stream, c->rw ? 0.234 : 0.65))
      return bfail(b, SMC_ERR_CUDA, "step size");
  }
  return SMC_OK;
}

int smc_batch_init(smc_batch **out, int32_t P, const smc_problem *probs, const smc_config *cfgs,
                   void *stream) {
  if (!out || P < 1 || !probs || !cfgs) return SMC_ERR_ARG;
  *out = nullptr;
  // one estimator tile for the whole batch: the narrowest compiled BF16 tile covering every row
  int need = 0;
  for (int q = 0; q < P; ++q) {
    if (probs[q].x_dtype != SMC_BF16) {
      g_init_error = "batches need BF16 storage";
      return SMC_ERR_ARG;
    }
    const int yo = ((probs[q].p * 2 + 15) / 16) * 8;
    if (yo > need) need = yo;
  }
  Tile tl[32];
  const int nt = est_tiles_bf16(tl, 32);
  int tile = -1;
  for (int t = 0; t < nt; ++t) {
    if (tl[t].T * tl[t].CPL < need) continue;
    const int wt = tl[t].T * tl[t].CPL, wb = tile < 0 ? 1 << 30 : tl[tile].T * tl[tile].CPL;
    if (wt < wb || (wt == wb && tl[t].T < tl[tile].T)) tile = t;
  }
  if (tile < 0) {
    g_init_error = "no compiled tile covers the batch's widest row";
    return SMC_ERR_ARG;
  }
  smc_batch *b = new smc_batch();
  b->P = P;
  b->tile = tile;
  b->stream = (cudaStream_t)stream;
  std::vector<int> off(P);
  for (int q = 0; q < P; ++q) {
    smc_config cfg = cfgs[q];
    cfg.tile_hint = tile + 1;
    cfg.hmc_kernel = 1;  // the context's own kernel; the batch chooses its trajectory launches
    cfg.full_data = 0;
    cfg.shard_base = cfg.shard_count = 0;
    smc_ctx *c = nullptr;
    const int r = smc_init(&c, &probs[q], &cfg, nullptr, stream);
    if (r != SMC_OK) {
      const std::string m = "problem " + std::to_string(q) + ": " + g_init_error;
      smc_batch_free(b);
      g_init_error = m;
      return r;
    }
    c->batch_member = true;
    b->ctx.push_back(c);
    off[q] = b->total;
    b->total += c->N;
    const int ws = est_warp_smem_bf16(tile, c->p);
    if (ws > b->wstride) b->wstride = ws;
  }
  if (cudaMalloc(&b->offsets_d, sizeof(int) * P) != cudaSuccess ||
      cudaMemcpy(b->offsets_d, off.data(), sizeof(int) * P, cudaMemcpyHostToDevice) != cudaSuccess) {
    smc_batch_free(b);
    g_init_error = "batch offsets";
    return SMC_ERR_OOM;
  }
  // groups: each problem goes to the narrowest resident tile that takes its p, m and G, with the
  // default warps per CTA for its p and m (res_default_warps; more when none fits), unless its
  // configuration asks for the streamed trajectory (hmc_kernel = 1)
  {
    static const int kCand4[][2] = {{0, 8},  {7, 12},  {1, 16},  {6, 20},
                                    {2, 24}, {3, 32},  {9, 40}};
    static const int kCand2[][2] = {{10, 8}, {11, 12}, {12, 16}, {13, 20},
                                    {14, 24}, {15, 32}, {16, 40}};
    static const int kCand1[][2] = {{17, 8}, {18, 12}, {19, 16}, {20, 20},
                                    {21, 24}, {22, 32}, {23, 40}};
    std::vector<int> gt(P, -1);
    BatchArgs dry{};
    for (int q = 0; q < P; ++q) {
      // the random-walk move runs on the streamed kernel only
      if (cfgs[q].hmc_kernel == 1 || cfgs[q].theta_move == 1) continue;
      const smc_ctx *c = b->ctx[q];
      for (int w = res_default_warps(c->p, c->m); w <= 4 && gt[q] < 0; w *= 2) {
        const int(*cand)[2] = w == 1 ? kCand1 : w == 2 ? kCand2 : kCand4;
        for (int t = 0; t < 7; ++t)
          if (c->p <= cand[t][1] && res_launch_batch_bf16(cand[t][0], dry, c->p, c->m, c->G,
                                                          b->stream, c->sms, true) == 0) {
            gt[q] = cand[t][0];
            break;
          }
      }
    }
    std::vector<int> tiles;
    for (int q = 0; q < P; ++q)
      if (std::find(tiles.begin(), tiles.end(), gt[q]) == tiles.end()) tiles.push_back(gt[q]);
    b->group_of.assign(P, 0);
    std::vector<int> goff(P, 0);
    for (int t : tiles) {
      BatchGroup g{t, (int)b->order.size(), 0, 0, 0, 0, 0};
      for (int q = 0; q < P; ++q) {
        if (gt[q] != t) continue;
        const smc_ctx *c = b->ctx[q];
        b->group_of[q] = (int)b->groups.size();
        goff[b->order.size()] = g.total;
        b->order.push_back(q);
        g.count += 1;
        g.total += c->N;
        g.pmax = std::max(g.pmax, c->p);
        g.mmax = std::max(g.mmax, c->m);
        g.Gmax = std::max(g.Gmax, c->G);
      }
      if (t >= 0 && res_launch_batch_bf16(t, dry, g.pmax, g.mmax, g.Gmax, b->stream,
                                          b->ctx[0]->sms, true) != 0) {
        smc_batch_free(b);
        g_init_error = "batch: a resident group's plan does not fit";
        return SMC_ERR_ARG;
      }
      b->groups.push_back(g);
    }
    if (cudaMalloc(&b->goff_d, sizeof(int) * P) != cudaSuccess ||
        cudaMemcpy(b->goff_d, goff.data(), sizeof(int) * P, cudaMemcpyHostToDevice) != cudaSuccess) {
      smc_batch_free(b);
      g_init_error = "batch group offsets";
      return SMC_ERR_OOM;
    }
  }
  // batched stage steps: every problem with a fixed centre (cv_centre = 0) and p <= 128
  b->stage_kernels = true;
  for (const smc_ctx *c : b->ctx)
    if (c->cv_centre != 0 || c->full_data || c->is_f64 || c->p > 128 || c->parity != 0)
      b->stage_kernels = false;
  if (b->stage_kernels) {
    std::vector<StageArgs> sa[2];
    std::vector<int> off((size_t)kSkKinds * (P + 1), 0);
    b->sb = StageBatch{};
    b->sb.P = P;
    for (int q = 0; q < P; ++q) {
      const smc_ctx *c = b->ctx[q];
      const bool grid = c->grid_points > 0;
      const int rounds = grid ? (c->grid_points + kSearchMaxK - 1) / kSearchMaxK : c->rounds;
      StageArgs a{};
      a.N = c->N;
      a.p = c->p;
      a.m = c->m;
      a.G = c->G;
      a.K = grid ? kSearchMaxK : c->K;
      a.last_round = rounds - 1;
      a.S = c->grid_points;
      a.multinomial = c->multinomial;
      a.tau = c->tau;
      a.E = c->grid_decades;
      a.eps_target = c->rw ? 0.234 : 0.65;
      a.seed = c->seed;
      a.st = c->st;
      a.part = c->part;
      a.logW = c->logW;
      a.W = c->W;
      a.mean = c->mean_d;
      a.Sigma_raw = c->Sigma_raw;
      a.Sigma = c->Sigma_d;
      a.chol = c->chol_d;
      a.work = c->mass_work;
      a.Sigma_ct = static_cast<float *>(c->Sigma_ct);
      a.Linv_ct = static_cast<float *>(c->Linv_ct);
      a.cum = c->cum;
      a.anc = c->anc;
      for (int par = 0; par < 2; ++par) {  // parity 0: the buffers current at init
        StageArgs t = a;
        float *th[2] = {static_cast<float *>(c->theta), static_cast<float *>(c->theta_alt)};
        int32_t *uu[2] = {c->u, c->u_alt};
        double *el[2] = {c->ell, c->ell_alt}, *sg[2] = {c->sig2, c->sig2_alt};
        double *bk[2] = {c->blk, c->blk_alt};
        t.theta = th[par];
        t.theta_out = th[par ^ 1];
        t.u = uu[par];
        t.u_out = uu[par ^ 1];
        t.ell = el[par];
        t.ell_out = el[par ^ 1];
        t.sig2 = sg[par];
        t.sig2_out = sg[par ^ 1];
        t.blk = bk[par];
        t.blk_out = bk[par ^ 1];
        sa[par].push_back(t);
      }
      for (int k = 0; k < kSkKinds; ++k)
        off[(size_t)k * (P + 1) + q + 1] =
            off[(size_t)k * (P + 1) + q] + stage_kind_blocks(k, c->N, c->p);
      b->sb.max_rounds = std::max(b->sb.max_rounds, rounds);
      b->sb.max_p = std::max(b->sb.max_p, c->p);
    }
    for (int k = 0; k < kSkKinds; ++k) b->sb.total[k] = off[(size_t)k * (P + 1) + P];
    bool ok = cudaMalloc(&b->soff_d, sizeof(int) * off.size()) == cudaSuccess &&
              cudaMemcpy(b->soff_d, off.data(), sizeof(int) * off.size(),
                         cudaMemcpyHostToDevice) == cudaSuccess;
    for (int par = 0; par < 2 && ok; ++par)
      ok = cudaMalloc(&b->sargs_d[par], sizeof(StageArgs) * P) == cudaSuccess &&
           cudaMemcpy(b->sargs_d[par], sa[par].data(), sizeof(StageArgs) * P,
                      cudaMemcpyHostToDevice) == cudaSuccess;
    if (!ok) {
      smc_batch_free(b);
      g_init_error = "batch stage arguments";
      return SMC_ERR_OOM;
    }
    b->sb.off = b->soff_d;
  }
  const int ns = P < 16 ? P : 16;
  b->side.assign(ns, nullptr);
  b->ev_side.assign(ns, nullptr);
  bool ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; k < ns && ok; ++k)
    ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&b->ev_side[k], cudaEventDisableTiming) == cudaSuccess;
  if (!ok) {
    smc_batch_free(b);
    g_init_error = "batch side streams";
    return SMC_ERR_CUDA;
  }
  *out = b;
  return SMC_OK;
}

int smc_batch_free(smc_batch *b) {
  if (!b) return SMC_OK;
  if (b->stream || !b->ctx.empty()) cudaStreamSynchronize(b->stream);
  for (int q = 0; q < 2; ++q) {
    if (b->gexec[q]) cudaGraphExecDestroy(b->gexec[q]);
    if (b->gargs[q]) cudaFree(b->gargs[q]);
  }
  for (smc_ctx *c : b->ctx) smc_free(c);
  if (b->offsets_d) cudaFree(b->offsets_d);
  if (b->goff_d) cudaFree(b->goff_d);
  if (b->soff_d) cudaFree(b->soff_d);
  for (StageArgs *a : b->sargs_d)
    if (a) cudaFree(a);
  if (b->args_d) cudaFree(b->args_d);
  for (cudaStream_t st : b->side)
    if (st) cudaStreamDestroy(st);
  for (cudaEvent_t e : b->ev_side)
    if (e) cudaEventDestroy(e);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  delete b;
  return SMC_OK;
}

const char *smc_batch_last_error(const smc_batch *b) {
  return b ? b->err.c_str() : g_init_error.c_str();
}

int smc_batch_context(smc_batch *b, int32_t q, smc_ctx **ctx) {
  if (!b || !ctx || q < 0 || q >= b->P) return SMC_ERR_ARG;
  *ctx = b->ctx[q];
  return SMC_OK;
}

int smc_batch_tile(const smc_batch *b, int32_t *tile_hint) {
  if (!b || !tile_hint) return SMC_ERR_ARG;
  *tile_hint = b->tile + 1;
  return SMC_OK;
}

int smc_batch_hmc_kernel(const smc_batch *b, int32_t q, int32_t *hmc_kernel) {
  if (!b || !hmc_kernel || q < 0 || q >= b->P) return SMC_ERR_ARG;
  const int t = b->groups[b->group_of[q]].tile;
  *hmc_kernel = t >= 0 ? t + 2 : 1;
  return SMC_OK;
}

int64_t smc_batch_launch_count(const smc_batch *b) {
  if (!b) return 0;
  int64_t n = b->launches;
  for (smc_ctx *c : b->ctx) n += c->launches;
  return n;
}

int smc_batch_stage(smc_batch *b, int32_t R, int32_t use_graph) {
  if (!b) return SMC_ERR_ARG;
  if (R < 1 || R > 256) return bfail(b, SMC_ERR_ARG, "R must be in [1, 256]");
  if (!use_graph) return batch_stage_body(b, R, false);
  const int q = b->ctx[0]->parity;
  for (smc_ctx *c : b->ctx) {
    if (c->parity != q) return bfail(b, SMC_ERR_STATE, "batch problems out of step");
    if (!c->dev_stage_synced) {
      if (stage_set(c->st, c->stage, b->stream)) return bfail(b, SMC_ERR_CUDA, "stage counter");
      c->dev_stage_synced = true;
    }
  }
  if (!(b->gexec[q] && b->gR[q] == R)) {
    if (b->gexec[q]) cudaGraphExecDestroy(b->gexec[q]);
    b->gexec[q] = nullptr;
    if (b->gargs[q]) cudaFree(b->gargs[q]);
    b->gargs[q] = nullptr;
    // arguments of this parity's graph: the buffers after the stage's resampling, stage index
    // from the device counters; kept in their own slot of the argument array
    int r = batch_upload(b, R, true, 1);
    if (r) return r;
    EstArgs *keep = b->args_d;  // becomes this graph's argument array
    b->gargs[q] = keep;
    b->args_d = nullptr;
    b->Rcap = 0;
    cudaStream_t cap;
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess)
      return bfail(b, SMC_ERR_CUDA, "capture stream");
    cudaStream_t orig = b->stream;
    cudaStreamSynchronize(orig);  // the argument upload has completed
    if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaStreamDestroy(cap);
      return bfail(b, SMC_ERR_CUDA, "batch capture");
    }
    int64_t l0 = b->launches;
    for (smc_ctx *c : b->ctx) l0 += c->launches;
    b->stream = cap;
    for (smc_ctx *c : b->ctx) {
      c->stream = cap;
      c->capturing = true;
      c->stage_dev = 1;
    }
    b->args_d = keep;
    b->Rcap = R;
    r = 0;
    if (!batch_stage_kernels(b))  // the batched stage steps advance the counters themselves
      for (smc_ctx *c : b->ctx)
        if (!r && stage_advance(c->st, cap)) r = SMC_ERR_CUDA;
    if (!r) r = batch_stage_body(b, R, true);
    cudaGraph_t g = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(cap, &g);
    b->stream = orig;
    for (smc_ctx *c : b->ctx) {
      c->stream = orig;
      c->capturing = false;
      c->stage_dev = 0;
    }
    cudaStreamDestroy(cap);
    // the capture consumed this argument array: the next upload gets a fresh one
    b->args_d = nullptr;
    b->Rcap = 0;
    if (r || e2 != cudaSuccess || !g) {
      if (g) cudaGraphDestroy(g);
      return r ? r : bfail(b, SMC_ERR_CUDA, std::string("batch capture: ") + cudaGetErrorString(e2));
    }
    const cudaError_t e3 = cudaGraphInstantiate(&b->gexec[q], g, 0);
    cudaGraphDestroy(g);
    if (e3 != cudaSuccess) {
      b->gexec[q] = nullptr;
      return bfail(b, SMC_ERR_CUDA, "batch graph instantiate");
    }
    b->gR[q] = R;
    {
      int64_t nl = b->launches;
      for (smc_ctx *c : b->ctx) nl += c->launches;
      b->glaunches[q] = nl - l0;
    }
    if (cudaGraphLaunch(b->gexec[q], b->stream) != cudaSuccess)
      return bfail(b, SMC_ERR_CUDA, "batch graph launch");
    return SMC_OK;  // capturing ran the host side of the stage; the launch runs its device side
  }
  if (cudaGraphLaunch(b->gexec[q], b->stream) != cudaSuccess)
    return bfail(b, SMC_ERR_CUDA, "batch graph launch");
  b->launches += b->glaunches[q];
  for (smc_ctx *c : b->ctx) {  // the host side of the replayed stage
    c->stage += 1;
    c->moves_in_stage = R;
    std::swap(c->theta, c->theta_alt);
    std::swap(c->u, c->u_alt);
    std::swap(c->ell, c->ell_alt);
    std::swap(c->sig2, c->sig2_alt);
    std::swap(c->blk, c->blk_alt);
    c->parity ^= 1;
  }
  return SMC_OK;
}

int smc_batch_autotune(smc_batch *b, int32_t *tile_hint) {
  if (!b) return SMC_ERR_ARG;
  int need = 0;
  for (smc_ctx *c : b->ctx)
    if (c->Sx > need) need = c->Sx;
  Tile tl[32];
  const int nt = est_tiles_bf16(tl, 32);
  // scratch copies: the batched HMC runs on theta_alt, ell_alt, sig2_alt, blk_alt
  b->args_h.resize(b->P);
  for (int q = 0; q < b->P; ++q) {
    smc_ctx *c = b->ctx[q];
    if (cudaMemcpyAsync(c->theta_alt, c->theta, ct_size(c) * c->N * c->p, cudaMemcpyDeviceToDevice,
                        b->stream) != cudaSuccess)
      return bfail(b, SMC_ERR_CUDA, "autotune copy");
    EstArgs a = batch_move_args(c, 255, false, 0);
    a.theta = a.theta_out = c->theta_alt;
    a.ell = c->ell_alt;
    a.sig2 = c->sig2_alt;
    a.blk = c->blk_alt;
    b->args_h[q] = a;
  }
  EstArgs *tmp = nullptr;
  if (cudaMalloc(&tmp, sizeof(EstArgs) * b->P) != cudaSuccess)
    return bfail(b, SMC_ERR_OOM, "autotune arguments");
  cudaMemcpyAsync(tmp, b->args_h.data(), sizeof(EstArgs) * b->P, cudaMemcpyHostToDevice, b->stream);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = b->tile;
  float best_ms = 1e30f;
  for (int t = 0; t < nt; ++t) {
    if (tl[t].T * tl[t].CPL < need) continue;
    int ws = 0;
    for (smc_ctx *c : b->ctx) ws = std::max(ws, est_warp_smem_bf16(t, c->p));
    BatchArgs ba{tmp, b->offsets_d, b->P, b->total, ws};
    float tot = 0.f;
    bool ok = true;
    for (int rep = 0; rep < 3 && ok; ++rep) {
      cudaEventRecord(e0, b->stream);
      ok = est_launch_batch_bf16(2, t, ba, b->stream) == 0;
      cudaEventRecord(e1, b->stream);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) tot += ms;  // the first run warms up
    }
    if (ok && tot < best_ms) {
      best_ms = tot;
      best = t;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(tmp);
  b->tile = best;
  b->wstride = 0;
  for (smc_ctx *c : b->ctx) {
    b->wstride = std::max(b->wstride, est_warp_smem_bf16(best, c->p));
    c->tile = best;
    cudaMemsetAsync(&c->st->acc_u, 0, 2 * sizeof(unsigned long long), b->stream);
  }
  for (int q = 0; q < 2; ++q) {  // graphs were built for the previous tile
    if (b->gexec[q]) cudaGraphExecDestroy(b->gexec[q]);
    if (b->gargs[q]) cudaFree(b->gargs[q]);
    b->gexec[q] = nullptr;
    b->gargs[q] = nullptr;
  }
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, SMC_ERR_CUDA, "autotune");
  if (tile_hint) *tile_hint = best + 1;
  return SMC_OK;
}

}  // extern "C"
