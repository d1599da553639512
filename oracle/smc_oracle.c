/*
 * Oracle for likelihood-annealed subsampling SMC (Gunawan, Dang, Quiroz, Kohn & Tran,
 * "Subsampling Sequential Monte Carlo for Static Bayesian Models", arXiv:1805.03317).
 *
 * TEST INFRASTRUCTURE ONLY. This file is a plain, slow, FP64 CPU restatement of the method, used
 * to check the CUDA library. Only the tests, the smoke check and the CPU-baseline leg of the
 * benchmark may load it; the product path never does. It shares no code, header, table or
 * constant generator with the CUDA library.
 *
 * Every routine follows the paper's definitions in their printed order, with no blocking, fusion
 * or reordering beyond what the definitions state:
 *   - per-row log-densities l_k(theta) of the GLM families            (Sec. 3.1, Eq. likelihood)
 *   - second-order Taylor control variates q_k and the moments A,B,C   (Sec. 3.2)
 *   - the difference estimator l_hat_m and its variance sigma2_hat_m   (Sec. 3.2, Eq. difference_estimator_logl)
 *   - the annealed likelihood estimator and the extended target        (Sec. 3.1, Eqs. tempered_likelihood_estimator,
 *                                                                       extended_target_at_sequence_p)
 *   - the block pseudo-marginal update of u and its MH ratio           (Algorithm 1 step 1, Eq. acc_prop_u)
 *   - the HMC move of theta given u, or a random-walk move             (Algorithm 1 step 2; Sec. 4.2)
 *   - first-order control variates                                     (Sec. 4, Experiment 4)
 *   - the Student-t regression family                                  (Sec. 4.3)
 *   - reweighting, ESS, tempering search, log marginal likelihood      (Sec. 2.2-2.3, Sec. 3.3, Sec. 3.5, Algorithm 2)
 *   - weighted moments / mass matrix and resampling                    (Algorithm 2 steps (d)-(e))
 *
 * Where the paper is silent the oracle takes these readings (the CUDA library takes the same ones):
 *   - random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11), counter
 *     (draw/2, particle, stage*256+move, tag), key (seed_lo, seed_hi); a 64-bit draw is two 32-bit
 *     outputs; an index in [0,n) is floor(r64*n/2^64); a uniform is (r64>>11)*2^-53; normals by
 *     Box-Muller (1958) with u1 = ((r64>>11)+1)*2^-53.
 *   - sigma2_hat_m is implemented as printed, (n^2/m^2) * sum_j (d_j - dbar)^2.
 *   - the HMC force is the exact gradient of a*l_hat - a^2/2*sigma2_hat + log p(theta) for fixed u.
 *   - u blocks are the contiguous floor partitions [floor(g*m/G), floor((g+1)*m/G)).
 *   - resampling is systematic, on weights quantised to integers floor(W_i * 2^40); the paper's
 *     multinomial scheme is the alternative, on the same integer weights.
 *   - the tempering increment is found by a K-ary refinement of a bracket (K=2 is bisection), or
 *     by the paper's grid rule on a geometric grid of increments.
 *   - each particle's HMC step is eps times a uniform on [1 - j, 1 + j] (j = 0.3 by default), drawn
 *     from the second word of its theta-MH Philox block; the random-walk scale is eps itself.
 *   - the Newton search for the posterior mode damps a Hessian that is not negative definite.
 *
 * Parity status per function: every exported function is pinned by the CPU tests (brute force,
 * enumeration, closed forms, published Philox vectors); see the test files.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { FAM_LOGISTIC = 0, FAM_PROBIT = 1, FAM_POISSON = 2, FAM_GAUSSIAN = 3, FAM_STUDENT_T = 4 };

/* Degrees of freedom nu of the Student-t family (Sec. 4.3: nu = 5). Process-wide; set by the Python
 * front end before each call, like the control-variate order below. */
static double g_dof = 5.0;
void orc_set_dof(double nu) { g_dof = nu; }
enum {
  TAG_INIT_THETA = 1, TAG_INIT_U = 2, TAG_UPM_BLOCK = 3, TAG_UPM_IDX = 4,
  TAG_MOMENTUM = 5, TAG_MH_THETA = 6, TAG_MH_U = 7, TAG_RESAMPLE = 8
};

/* ------------------------------------------------------------------------------------------ */
/* Philox4x32-10, written from its published definition (Salmon et al. 2011, Sec. 4 and        */
/* Table 2): ten rounds of two 32x32->64 multiplies, key bumped by the Weyl constants.           */
/* ------------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t *ctr, const uint32_t *key, uint32_t *out) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
    uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
    uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* j-th 64-bit draw of the stream (tag, stage*256+move, particle) under key seed. */
uint64_t orc_r64(uint64_t seed, uint32_t tag, uint32_t stage_move, uint32_t particle, uint64_t j) {
  uint32_t ctr[4] = {(uint32_t)(j >> 1), particle, stage_move, tag};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t o[4];
  orc_philox4x32_10(ctr, key, o);
  int h = (int)(j & 1);
  return ((uint64_t)o[2 * h + 1] << 32) | (uint64_t)o[2 * h];
}

/* Index uniform on {0..n-1}: floor(r64 * n / 2^64), exact in 128-bit arithmetic. */
int64_t orc_index(uint64_t r64, int64_t n) {
  return (int64_t)(((unsigned __int128)r64 * (unsigned __int128)(uint64_t)n) >> 64);
}

/* Uniform on [0,1) with 53 random bits. */
double orc_uniform(uint64_t r64) { return (double)(r64 >> 11) * 0x1.0p-53; }

/* j-th standard normal of a stream: Box-Muller on the two 64-bit draws of Philox block j/2. */
double orc_normal(uint64_t seed, uint32_t tag, uint32_t stage_move, uint32_t particle, uint64_t j) {
  uint64_t blk = j >> 1;
  uint64_t ra = orc_r64(seed, tag, stage_move, particle, 2 * blk);
  uint64_t rb = orc_r64(seed, tag, stage_move, particle, 2 * blk + 1);
  double u1 = (double)((ra >> 11) + 1) * 0x1.0p-53; /* (0,1] */
  double u2 = (double)(rb >> 11) * 0x1.0p-53;       /* [0,1) */
  double r = sqrt(-2.0 * log(u1));
  const double two_pi = 6.283185307179586476925286766559;
  return (j & 1) ? r * sin(two_pi * u2) : r * cos(two_pi * u2);
}

/* ------------------------------------------------------------------------------------------ */
/* Per-row log-density l_k = log p(y_k | theta) of the GLM families and its first and second     */
/* derivatives in the linear predictor eta = x_k' theta (Sec. 3.1, Eq. likelihood; logistic in    */
/* Sec. 4.2, Poisson in Sec. 4.3; Gaussian and probit as used by the synthetic workloads).        */
/* ------------------------------------------------------------------------------------------ */

/* erfcx(x) = exp(x^2) erfc(x) for x >= 3, by Laplace's continued fraction
 *   erfc(x) = exp(-x^2)/sqrt(pi) * 1/(x + (1/2)/(x + 1/(x + (3/2)/(x + 2/(x + ...)))))
 * evaluated bottom-up with 80 terms. */
double orc_erfcx_cf(double x) {
  double t = x;
  for (int k = 80; k >= 1; --k) t = x + (0.5 * k) / t;
  return 1.0 / (t * 1.7724538509055160272981674833411);
}

/* log Phi(z) and the inverse Mills ratio lambda(z) = phi(z)/Phi(z). */
static void orc_log_phi(double z, double *logphi, double *lambda) {
  const double inv_sqrt2 = 0.70710678118654752440084436210485;
  const double sqrt_2_over_pi = 0.79788456080286535587989211986876;
  double x = -z * inv_sqrt2;
  if (x < 3.0) {
    double Phi = 0.5 * erfc(x);
    double phi = exp(-0.5 * z * z) * 0.39894228040143267793994605993438;
    *logphi = log(Phi);
    *lambda = phi / Phi;
  } else {
    double ex = orc_erfcx_cf(x);
    *logphi = log(0.5 * ex) - x * x;
    *lambda = sqrt_2_over_pi / ex;
  }
}

void orc_family(int fam, double eta, double y, double sigma, double *l, double *d1, double *d2) {
  switch (fam) {
    case FAM_LOGISTIC: {
      /* l = y*eta - log(1 + e^eta) */
      double softplus = eta > 0 ? eta + log1p(exp(-eta)) : log1p(exp(eta));
      double s = 1.0 / (1.0 + exp(-eta));
      *l = y * eta - softplus;
      *d1 = y - s;
      *d2 = -s * (1.0 - s);
      break;
    }
    case FAM_POISSON: {
      /* l = y*eta - e^eta - log(y!) */
      double mu = exp(eta);
      *l = y * eta - mu - lgamma(y + 1.0);
      *d1 = y - mu;
      *d2 = -mu;
      break;
    }
    case FAM_GAUSSIAN: {
      /* l = -log(2 pi sigma^2)/2 - (y - eta)^2 / (2 sigma^2) */
      double s2 = sigma * sigma, r = y - eta;
      *l = -0.5 * log(6.283185307179586476925286766559 * s2) - r * r / (2.0 * s2);
      *d1 = r / s2;
      *d2 = -1.0 / s2;
      break;
    }
    case FAM_STUDENT_T: {
      /* y = eta + s*e, e ~ t_nu (Sec. 4.3): l = log Gamma((nu+1)/2) - log Gamma(nu/2)
       * - log(nu pi s^2)/2 - (nu+1)/2 log(1 + (y - eta)^2 / (nu s^2)) */
      double nu = g_dof, s2 = sigma * sigma, r = y - eta, q = nu * s2 + r * r;
      *l = lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) - 0.5 * log(3.14159265358979323846 * nu * s2) -
           0.5 * (nu + 1.0) * log(q / (nu * s2));
      *d1 = (nu + 1.0) * r / q;
      *d2 = (nu + 1.0) * (r * r - nu * s2) / (q * q);
      break;
    }
    case FAM_PROBIT: {
      /* l = log Phi(s*eta), s = 2y - 1 */
      double s = 2.0 * y - 1.0, z = s * eta, lp, lam;
      orc_log_phi(z, &lp, &lam);
      *l = lp;
      *d1 = s * lam;
      *d2 = -lam * (z + lam);
      break;
    }
    default:
      *l = *d1 = *d2 = NAN;
  }
}

static double dot(const double *a, const double *b, int p) {
  double s = 0.0;
  for (int c = 0; c < p; ++c) s += a[c] * b[c];
  return s;
}

/* Full-data log-likelihood l(theta) = sum_k l_k(theta) and its gradient (Eq. likelihood). */
void orc_full_loglik(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                     const double *theta, double *ell, double *grad) {
  double L = 0.0;
  if (grad) memset(grad, 0, sizeof(double) * p);
  for (int64_t k = 0; k < n; ++k) {
    const double *x = X + k * p;
    double l, d1, d2;
    orc_family(fam, dot(x, theta, p), y[k], sigma, &l, &d1, &d2);
    L += l;
    if (grad)
      for (int c = 0; c < p; ++c) grad[c] += d1 * x[c];
  }
  *ell = L;
}

/* Control-variate moments at theta_bar (Sec. 3.2):
 *   A = sum_k l_k(theta_bar),  B = sum_k grad l_k(theta_bar),  C = sum_k hess l_k(theta_bar).
 * For a GLM, grad l_k = l'(eta_bar) x_k and hess l_k = l''(eta_bar) x_k x_k'. Direct sums over k. */
void orc_cv_moments(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                    const double *theta_bar, double *A, double *B, double *C) {
  double a = 0.0;
  memset(B, 0, sizeof(double) * p);
  memset(C, 0, sizeof(double) * p * p);
  for (int64_t k = 0; k < n; ++k) {
    const double *x = X + k * p;
    double l, d1, d2;
    orc_family(fam, dot(x, theta_bar, p), y[k], sigma, &l, &d1, &d2);
    a += l;
    for (int r = 0; r < p; ++r) {
      B[r] += d1 * x[r];
      for (int c = 0; c < p; ++c) C[r * p + c] += d2 * x[r] * x[c];
    }
  }
  *A = a;
}

/* Diagonal Gaussian prior N(mu, diag(v)): log density and gradient. */
double orc_log_prior(int p, const double *theta, const double *mu, const double *v, double *grad) {
  double lp = 0.0;
  for (int c = 0; c < p; ++c) {
    double r = theta[c] - mu[c];
    lp += -0.5 * r * r / v[c] - 0.5 * log(6.283185307179586476925286766559 * v[c]);
    if (grad) grad[c] = -r / v[c];
  }
  return lp;
}

/* Everything the subsampled estimator needs about the problem. */
typedef struct {
  int fam;
  int64_t n;
  int p;
  const double *X; /* [n,p] */
  const double *y; /* [n]   */
  double sigma;    /* Gaussian noise sd, Student-t scale */
  const double *theta_bar, *B, *C;
  double A;
  const double *prior_mu, *prior_var;
  int m, G;
} orc_prob;

static int64_t block_start(int g, int m, int G) { return ((int64_t)g * m) / G; }

/* Order of the Taylor control variate: 2 (q_k to second order, the paper's main estimator) or 1
 * (first order: q_k = l_k(tb) + grad l_k(tb)'delta; Sec. 4's first-order variant). Process-wide;
 * set by the Python front end before each call. */
static int g_cv_order = 2;
void orc_set_cv_order(int k) { g_cv_order = (k == 1) ? 1 : 2; }

/* Difference estimator (Sec. 3.2, Eq. difference_estimator_logl) for one particle:
 *   l_hat = sum_k q_k(theta) + (n/m) sum_j [l_{u_j}(theta) - q_{u_j}(theta)]
 *   sigma2_hat = (n^2/m^2) sum_j (d_{u_j} - dbar)^2,  d_k = l_k - q_k
 * with q_k the second-order Taylor expansion of l_k around theta_bar, and sum_k q_k = A + B'delta +
 * delta'C delta / 2. Optionally the gradient of the annealed log target
 *   a*l_hat - (a^2/2)*sigma2_hat + log p(theta)     (Eq. extended_target_at_sequence_p)
 * for fixed u, and the per-block sums (sum d, sum d^2) over the floor partition of u into G blocks. */
void orc_loglik_one(const orc_prob *P, const int64_t *u, const double *theta, double a,
                    double *ell, double *sig2, double *grad, double *blk) {
  int p = P->p, m = P->m;
  double n = (double)P->n;
  double *delta = (double *)malloc(sizeof(double) * p);
  double *dvals = (double *)malloc(sizeof(double) * m);
  double *rvals = (double *)malloc(sizeof(double) * m);
  for (int c = 0; c < p; ++c) delta[c] = theta[c] - P->theta_bar[c];

  /* sum_k q_k(theta) = A + B'delta + (1/2) delta'C delta (first order: A + B'delta) */
  const double c2 = g_cv_order == 2 ? 1.0 : 0.0;
  double q_total = P->A;
  for (int r = 0; r < p; ++r) {
    q_total += P->B[r] * delta[r];
    for (int c = 0; c < p; ++c) q_total += c2 * 0.5 * delta[r] * P->C[r * p + c] * delta[c];
  }

  double dsum = 0.0;
  for (int j = 0; j < m; ++j) {
    const double *x = P->X + u[j] * p;
    double l, d1, d2, lb, d1b, d2b;
    double eta = dot(x, theta, p), eta_bar = dot(x, P->theta_bar, p);
    orc_family(P->fam, eta, P->y[u[j]], P->sigma, &l, &d1, &d2);
    orc_family(P->fam, eta_bar, P->y[u[j]], P->sigma, &lb, &d1b, &d2b);
    /* q_k(theta) = l_k(tb) + grad l_k(tb)'delta + delta' hess l_k(tb) delta / 2 */
    double xd = dot(x, delta, p);
    double q = lb + d1b * xd + c2 * 0.5 * d2b * xd * xd;
    dvals[j] = l - q;
    /* d/dtheta d_k = [l'(eta) - l'(eta_bar) - l''(eta_bar) x'delta] x_k (no last term at first
     * order) */
    rvals[j] = d1 - d1b - c2 * d2b * xd;
    dsum += dvals[j];
  }
  double dbar = dsum / m;
  double ss = 0.0;
  for (int j = 0; j < m; ++j) ss += (dvals[j] - dbar) * (dvals[j] - dbar);

  *ell = q_total + (n / m) * dsum;
  *sig2 = (n * n) / ((double)m * m) * ss;

  if (blk) {
    for (int g = 0; g < P->G; ++g) {
      double s = 0.0, s2 = 0.0;
      for (int64_t j = block_start(g, m, P->G); j < block_start(g + 1, m, P->G); ++j) {
        s += dvals[j];
        s2 += dvals[j] * dvals[j];
      }
      blk[2 * g] = s;
      blk[2 * g + 1] = s2;
    }
  }

  if (grad) {
    /* grad l_hat = B + C delta + (n/m) sum_j r_j x_j
     * grad sigma2_hat = (n^2/m^2) * 2 * sum_j (d_j - dbar) r_j x_j */
    double *gl = (double *)calloc(p, sizeof(double));
    double *gs = (double *)calloc(p, sizeof(double));
    for (int r = 0; r < p; ++r) {
      gl[r] = P->B[r];
      for (int c = 0; c < p; ++c) gl[r] += c2 * P->C[r * p + c] * delta[c];
    }
    for (int j = 0; j < m; ++j) {
      const double *x = P->X + u[j] * p;
      for (int c = 0; c < p; ++c) {
        gl[c] += (n / m) * rvals[j] * x[c];
        gs[c] += (n * n) / ((double)m * m) * 2.0 * (dvals[j] - dbar) * rvals[j] * x[c];
      }
    }
    double *gp = (double *)malloc(sizeof(double) * p);
    orc_log_prior(p, theta, P->prior_mu, P->prior_var, gp);
    for (int c = 0; c < p; ++c) grad[c] = a * gl[c] - 0.5 * a * a * gs[c] + gp[c];
    free(gl);
    free(gs);
    free(gp);
  }
  free(delta);
  free(dvals);
  free(rvals);
}

static orc_prob make_prob(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                          const double *tb, double A, const double *B, const double *C,
                          const double *pm, const double *pv, int m, int G) {
  orc_prob P;
  P.fam = fam; P.n = n; P.p = p; P.X = X; P.y = y; P.sigma = sigma;
  P.theta_bar = tb; P.A = A; P.B = B; P.C = C; P.prior_mu = pm; P.prior_var = pv;
  P.m = m; P.G = G;
  return P;
}

/* Batch of particles: thetas [Bn,p], us [Bn,m] int64; outputs ell, sig2 [Bn], grad [Bn,p] or NULL,
 * blk [Bn,G,2] or NULL. */
void orc_loglik_batch(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                      const double *tb, double A, const double *B, const double *C,
                      const double *pm, const double *pv, int m, int G, int Bn,
                      const double *thetas, const int64_t *us, double a, double *ell, double *sig2,
                      double *grad, double *blk) {
  orc_prob P = make_prob(fam, n, p, X, y, sigma, tb, A, B, C, pm, pv, m, G);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < Bn; ++i)
    orc_loglik_one(&P, us + (int64_t)i * m, thetas + (int64_t)i * p, a, ell + i, sig2 + i,
                   grad ? grad + (int64_t)i * p : NULL, blk ? blk + (int64_t)i * G * 2 : NULL);
}

/* Annealed log target at (theta, u) (Eq. extended_target_at_sequence_p, up to log p(u)). */
static double log_target(const orc_prob *P, const int64_t *u, const double *theta, double a,
                         double *grad) {
  double ell, s2;
  orc_loglik_one(P, u, theta, a, &ell, &s2, grad, NULL);
  return a * ell - 0.5 * a * a * s2 + orc_log_prior(P->p, theta, P->prior_mu, P->prior_var, NULL);
}

/* ------------------------------------------------------------------------------------------ */
/* Initialisation (Algorithm 2 step 1): theta ~ prior, u ~ p(u) (iid uniform, with replacement).  */
/* ------------------------------------------------------------------------------------------ */
void orc_init(uint64_t seed, int N, int p, int m, int64_t n, const double *pm, const double *pv,
              double *thetas, int64_t *us) {
  for (int i = 0; i < N; ++i) {
    for (int c = 0; c < p; ++c)
      thetas[(int64_t)i * p + c] =
          pm[c] + sqrt(pv[c]) * orc_normal(seed, TAG_INIT_THETA, 0, (uint32_t)i, (uint64_t)c);
    for (int j = 0; j < m; ++j)
      us[(int64_t)i * m + j] = orc_index(orc_r64(seed, TAG_INIT_U, 0, (uint32_t)i, (uint64_t)j), n);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Optional record of every MH decision of the moves below: margin[i] = log ratio - log U of       */
/* particle i (> 0: accepted). Test support only: a caller that computes the same ratio in lower  */
/* precision may decide differently only where this margin is within its rounding. NULL = off.    */
/* ------------------------------------------------------------------------------------------ */
static double *g_margin = NULL;
void orc_set_margin_out(double *buf) { g_margin = buf; }

/* ------------------------------------------------------------------------------------------ */
/* Block pseudo-marginal update of u (Algorithm 1 step 1, Eq. acc_prop_u): one block g of the G   */
/* blocks is chosen uniformly, its indices are redrawn iid from p(u), and the proposal is          */
/* accepted with probability min(1, r), r the ratio of annealed likelihood estimators at theta.     */
/* us is updated in place; accepted[i] = 1 on acceptance.                                          */
/* ------------------------------------------------------------------------------------------ */
void orc_upm_move(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                  const double *tb, double A, const double *B, const double *C, const double *pm,
                  const double *pv, int m, int G, int N, uint64_t seed, uint32_t stage_move,
                  double a, const double *thetas, int64_t *us, int *accepted) {
  orc_prob P = make_prob(fam, n, p, X, y, sigma, tb, A, B, C, pm, pv, m, G);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < N; ++i) {
    int64_t *u = us + (int64_t)i * m;
    const double *theta = thetas + (int64_t)i * p;
    int64_t *ustar = (int64_t *)malloc(sizeof(int64_t) * m);
    memcpy(ustar, u, sizeof(int64_t) * m);
    int g = (int)orc_index(orc_r64(seed, TAG_UPM_BLOCK, stage_move, (uint32_t)i, 0), G);
    int64_t b0 = block_start(g, m, G), b1 = block_start(g + 1, m, G);
    for (int64_t j = b0; j < b1; ++j)
      ustar[j] = orc_index(orc_r64(seed, TAG_UPM_IDX, stage_move, (uint32_t)i, (uint64_t)(j - b0)), n);
    double ell, s2, ells, s2s;
    orc_loglik_one(&P, u, theta, a, &ell, &s2, NULL, NULL);
    orc_loglik_one(&P, ustar, theta, a, &ells, &s2s, NULL, NULL);
    double log_r = (a * ells - 0.5 * a * a * s2s) - (a * ell - 0.5 * a * a * s2);
    double U = orc_uniform(orc_r64(seed, TAG_MH_U, stage_move, (uint32_t)i, 0));
    int acc = log(U) < log_r;
    if (g_margin) g_margin[i] = log_r - log(U);
    if (acc) memcpy(u, ustar, sizeof(int64_t) * m);
    accepted[i] = acc;
    free(ustar);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Lsteps leapfrog steps of size eps for the Hamiltonian -log target(theta) + rho' Sigma rho / 2  */
/* at fixed u (Algorithm 1 step 2): half kick with the gradient, drift by eps Sigma rho, gradient */
/* at the new point, half kick. On entry g holds the gradient at th and lt the log target there; */
/* th, rho and g are updated in place, v is scratch [p]. Returns the log target at the end.       */
/* ------------------------------------------------------------------------------------------ */
static double leapfrog(const orc_prob *P, const int64_t *u, double a, double eps, int Lsteps,
                       const double *Sigma, double *th, double *rho, double *g, double *v,
                       double lt) {
  const int p = P->p;
  for (int l = 0; l < Lsteps; ++l) {
    for (int c = 0; c < p; ++c) rho[c] += 0.5 * eps * g[c];
    for (int r = 0; r < p; ++r) {
      v[r] = 0.0;
      for (int c = 0; c < p; ++c) v[r] += Sigma[r * p + c] * rho[c];
    }
    for (int c = 0; c < p; ++c) th[c] += eps * v[c];
    lt = log_target(P, u, th, a, g);
    for (int c = 0; c < p; ++c) rho[c] += 0.5 * eps * g[c];
  }
  return lt;
}

/* Test support: one trajectory of the leapfrog above from (theta, rho), both updated in place;
 * returns the log target at the end point. */
double orc_leapfrog(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                    const double *tb, double A, const double *B, const double *C, const double *pm,
                    const double *pv, int m, int G, const int64_t *u, double a, double eps,
                    int Lsteps, const double *Sigma, double *theta, double *rho) {
  orc_prob P = make_prob(fam, n, p, X, y, sigma, tb, A, B, C, pm, pv, m, G);
  double *g = (double *)malloc(sizeof(double) * p);
  double *v = (double *)malloc(sizeof(double) * p);
  double lt = log_target(&P, u, theta, a, g);
  lt = leapfrog(&P, u, a, eps, Lsteps, Sigma, theta, rho, g, v, lt);
  free(g);
  free(v);
  return lt;
}

/* ------------------------------------------------------------------------------------------ */
/* HMC move of theta given u (Algorithm 1 step 2): momentum rho ~ N(0, H) with mass matrix         */
/* H = Sigma^{-1} (Algorithm 2 step (d)), drawn as rho = L^{-T} z with Sigma = L L'; L leapfrog     */
/* steps of size eps on the annealed log target; MH accept with the Hamiltonian difference.       */
/* Sigma [p,p] and its lower Cholesky factor Lc [p,p] are inputs. thetas updated in place.          */
/* ------------------------------------------------------------------------------------------ */
void orc_hmc_move(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                  const double *tb, double A, const double *B, const double *C, const double *pm,
                  const double *pv, int m, int G, int N, uint64_t seed, uint32_t stage_move,
                  double a, double eps, double jitter, int Lsteps, const double *Sigma,
                  const double *Lc, double *thetas, const int64_t *us, int *accepted) {
  orc_prob P = make_prob(fam, n, p, X, y, sigma, tb, A, B, C, pm, pv, m, G);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < N; ++i) {
    double *theta0 = thetas + (int64_t)i * p;
    const int64_t *u = us + (int64_t)i * m;
    double *z = (double *)malloc(sizeof(double) * p);
    double *rho = (double *)malloc(sizeof(double) * p);
    double *th = (double *)malloc(sizeof(double) * p);
    double *g = (double *)malloc(sizeof(double) * p);
    double *v = (double *)malloc(sizeof(double) * p);
    for (int c = 0; c < p; ++c)
      z[c] = orc_normal(seed, TAG_MOMENTUM, stage_move, (uint32_t)i, (uint64_t)c);
    /* back substitution: L' rho = z */
    for (int r = p - 1; r >= 0; --r) {
      double s = z[r];
      for (int c = r + 1; c < p; ++c) s -= Lc[c * p + r] * rho[c];
      rho[r] = s / Lc[r * p + r];
    }
    double kin0 = 0.0;
    for (int r = 0; r < p; ++r)
      for (int c = 0; c < p; ++c) kin0 += 0.5 * rho[r] * Sigma[r * p + c] * rho[c];
    memcpy(th, theta0, sizeof(double) * p);
    double lt0 = log_target(&P, u, th, a, g);
    double H0 = -lt0 + kin0;
    double lt = lt0;
    /* the particle's step size, uniform on [eps (1 - jitter), eps (1 + jitter)] (the second word
       of its theta-MH block): a random step size breaks the near-periodic trajectories of a fixed
       eps L on near-Gaussian targets (Neal 2011) */
    double eps_i = eps;
    if (jitter > 0.0) {
      double Uj = orc_uniform(orc_r64(seed, TAG_MH_THETA, stage_move, (uint32_t)i, 1));
      eps_i = eps * (1.0 - jitter + 2.0 * jitter * Uj);
    }
    lt = leapfrog(&P, u, a, eps_i, Lsteps, Sigma, th, rho, g, v, lt);
    double kin1 = 0.0;
    for (int r = 0; r < p; ++r)
      for (int c = 0; c < p; ++c) kin1 += 0.5 * rho[r] * Sigma[r * p + c] * rho[c];
    double H1 = -lt + kin1;
    double U = orc_uniform(orc_r64(seed, TAG_MH_THETA, stage_move, (uint32_t)i, 0));
    int acc = log(U) < H0 - H1;
    if (g_margin) g_margin[i] = (H0 - H1) - log(U);
    if (acc) memcpy(theta0, th, sizeof(double) * p);
    accepted[i] = acc;
    free(z); free(rho); free(th); free(g); free(v);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Random-walk Metropolis move of theta given u (the RW kernel of Sec. 4.2's comparison):         */
/*   theta* = theta + eps * Lc z,  z ~ N(0, I) (the momentum stream's normals), Sigma = Lc Lc',    */
/*   accepted when log U < log target(theta*) - log target(theta) (U from the theta-MH stream).   */
/* ------------------------------------------------------------------------------------------ */
void orc_rw_move(int fam, int64_t n, int p, const double *X, const double *y, double sigma,
                 const double *tb, double A, const double *B, const double *C, const double *pm,
                 const double *pv, int m, int G, int N, uint64_t seed, uint32_t stage_move,
                 double a, double eps, const double *Lc, double *thetas, const int64_t *us,
                 int *accepted) {
  orc_prob P = make_prob(fam, n, p, X, y, sigma, tb, A, B, C, pm, pv, m, G);
#pragma omp parallel for schedule(dynamic, 1)
  for (int i = 0; i < N; ++i) {
    double *theta0 = thetas + (int64_t)i * p;
    const int64_t *u = us + (int64_t)i * m;
    double *z = (double *)malloc(sizeof(double) * p);
    double *th = (double *)malloc(sizeof(double) * p);
    for (int c = 0; c < p; ++c)
      z[c] = orc_normal(seed, TAG_MOMENTUM, stage_move, (uint32_t)i, (uint64_t)c);
    for (int r = 0; r < p; ++r) {
      double s = 0.0;
      for (int c = 0; c <= r; ++c) s += Lc[r * p + c] * z[c];
      th[r] = theta0[r] + eps * s;
    }
    double lt0 = log_target(&P, u, theta0, a, NULL);
    double lt1 = log_target(&P, u, th, a, NULL);
    double U = orc_uniform(orc_r64(seed, TAG_MH_THETA, stage_move, (uint32_t)i, 0));
    int acc = log(U) < lt1 - lt0;
    if (g_margin) g_margin[i] = (lt1 - lt0) - log(U);
    if (acc) memcpy(theta0, th, sizeof(double) * p);
    accepted[i] = acc;
    free(z);
    free(th);
  }
}

/* ------------------------------------------------------------------------------------------ */
/* Reweighting with an adaptively chosen temperature (Sec. 2.2, Sec. 3.3, Algorithm 2 (b)-(c)).   */
/*   lw_i(D) = log W_i + D*l_hat_i - ((a+D)^2 - a^2)/2 * sigma2_hat_i                               */
/*   ESS(D)  = (sum_i e^{lw_i})^2 / sum_i e^{2 lw_i}                                                */
/* If ESS(1-a) >= tau*N the next temperature is 1. Otherwise a bracket [lo,hi] with ESS(lo) >=     */
/* tau*N > ESS(hi) is refined for `rounds` rounds: the K-1 interior points lo + (hi-lo)k/K are     */
/* evaluated and the bracket becomes the first sub-interval whose right end has ESS < tau*N.       */
/* The increment is lo (hi if lo is still 0). Returns the new temperature; log W is overwritten by  */
/* the normalised new log weights, W by their exponentials; *log_z_inc is the log of             */
/* sum_i W_i^{old} gamma_i (Sec. 3.5), *ess the ESS at the chosen increment.                      */
/* ------------------------------------------------------------------------------------------ */
static double lse(const double *v, int N) {
  double mx = -INFINITY;
  for (int i = 0; i < N; ++i) if (v[i] > mx) mx = v[i];
  if (!(mx > -INFINITY)) return mx;
  double s = 0.0;
  for (int i = 0; i < N; ++i) s += exp(v[i] - mx);
  return mx + log(s);
}

double orc_ess_at(int N, const double *logW, const double *ell, const double *sig2, double a,
                  double D) {
  double *lw = (double *)malloc(sizeof(double) * N);
  double *lw2 = (double *)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i) {
    lw[i] = logW[i] + D * ell[i] - 0.5 * ((a + D) * (a + D) - a * a) * sig2[i];
    lw2[i] = 2.0 * lw[i];
  }
  double e = exp(2.0 * lse(lw, N) - lse(lw2, N));
  free(lw);
  free(lw2);
  return e;
}

double orc_reweight(int N, double *logW, double *W, const double *ell, const double *sig2,
                    double a, double tau, int K, int rounds, double *log_z_inc, double *ess) {
  double target = tau * (double)N;
  double Dmax = 1.0 - a, D;
  if (orc_ess_at(N, logW, ell, sig2, a, Dmax) >= target) {
    D = Dmax;
  } else {
    double lo = 0.0, hi = Dmax;
    for (int r = 0; r < rounds; ++r) {
      int k;
      for (k = 1; k < K; ++k)
        if (orc_ess_at(N, logW, ell, sig2, a, lo + (hi - lo) * k / K) < target) break;
      double nlo = lo + (hi - lo) * (k - 1) / K;
      double nhi = (k < K) ? lo + (hi - lo) * k / K : hi;
      lo = nlo;
      hi = nhi;
    }
    D = lo > 0.0 ? lo : hi;
  }
  double a_new = (D == Dmax) ? 1.0 : a + D;
  double *lw = (double *)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i)
    lw[i] = logW[i] + D * ell[i] - 0.5 * ((a + D) * (a + D) - a * a) * sig2[i];
  double lse_new = lse(lw, N), lse_old = lse(logW, N);
  *log_z_inc = lse_new - lse_old;
  *ess = orc_ess_at(N, logW, ell, sig2, a, D);
  for (int i = 0; i < N; ++i) {
    logW[i] = lw[i] - lse_new;
    W[i] = exp(logW[i]);
  }
  free(lw);
  return a_new;
}

/* ------------------------------------------------------------------------------------------ */
/* The paper's grid rule for the next temperature (Sec. 2.3): ESS is evaluated at S grid points   */
/* and the point whose ESS is closest to tau*N is taken. Reading for the grid, which the paper    */
/* leaves open: increments D_s = (1-a) * 10^(-E*(S-1-s)/(S-1)), s = 0..S-1 (geometric, the last   */
/* point 1-a itself), scanned in ascending order so that a tie keeps the smaller increment.       */
/* Outputs as for orc_reweight.                                                                    */
/* ------------------------------------------------------------------------------------------ */
double orc_reweight_grid(int N, double *logW, double *W, const double *ell, const double *sig2,
                         double a, double tau, int S, double E, double *log_z_inc, double *ess) {
  double target = tau * (double)N;
  double Dmax = 1.0 - a;
  double best = INFINITY, D = Dmax;
  for (int s = 0; s < S; ++s) {
    double Ds = (s == S - 1) ? Dmax : Dmax * pow(10.0, -E * (double)(S - 1 - s) / (double)(S - 1));
    double dist = fabs(orc_ess_at(N, logW, ell, sig2, a, Ds) - target);
    if (dist < best) {
      best = dist;
      D = Ds;
    }
  }
  double a_new = (D == Dmax) ? 1.0 : a + D;
  double *lw = (double *)malloc(sizeof(double) * N);
  for (int i = 0; i < N; ++i)
    lw[i] = logW[i] + D * ell[i] - 0.5 * ((a + D) * (a + D) - a * a) * sig2[i];
  double lse_new = lse(lw, N), lse_old = lse(logW, N);
  *log_z_inc = lse_new - lse_old;
  *ess = orc_ess_at(N, logW, ell, sig2, a, D);
  for (int i = 0; i < N; ++i) {
    logW[i] = lw[i] - lse_new;
    W[i] = exp(logW[i]);
  }
  free(lw);
  return a_new;
}

/* ------------------------------------------------------------------------------------------ */
/* Weighted particle moments and the mass matrix (Algorithm 2 step (d)): mean = sum_i W_i theta_i, */
/* Sigma = sum_i W_i (theta_i - mean)(theta_i - mean)', and its lower Cholesky factor; if the      */
/* factorisation fails, jitter 1e-10*tr(Sigma)/p (times 10 per retry) is added to the diagonal.    */
/* Returns the number of jitter retries, or -1 if none succeeded.                                  */
/* ------------------------------------------------------------------------------------------ */
int orc_cholesky(int p, const double *S, double *Lc) {
  memset(Lc, 0, sizeof(double) * p * p);
  for (int j = 0; j < p; ++j) {
    double s = S[j * p + j];
    for (int k = 0; k < j; ++k) s -= Lc[j * p + k] * Lc[j * p + k];
    if (!(s > 0.0)) return -1;
    Lc[j * p + j] = sqrt(s);
    for (int i = j + 1; i < p; ++i) {
      double t = S[i * p + j];
      for (int k = 0; k < j; ++k) t -= Lc[i * p + k] * Lc[j * p + k];
      Lc[i * p + j] = t / Lc[j * p + j];
    }
  }
  return 0;
}

int orc_moments(int N, int p, const double *W, const double *thetas, double *mean, double *Sigma,
                double *Lc) {
  memset(mean, 0, sizeof(double) * p);
  memset(Sigma, 0, sizeof(double) * p * p);
  for (int i = 0; i < N; ++i)
    for (int c = 0; c < p; ++c) mean[c] += W[i] * thetas[(int64_t)i * p + c];
  for (int i = 0; i < N; ++i)
    for (int r = 0; r < p; ++r)
      for (int c = 0; c < p; ++c)
        Sigma[r * p + c] += W[i] * (thetas[(int64_t)i * p + r] - mean[r]) *
                            (thetas[(int64_t)i * p + c] - mean[c]);
  if (orc_cholesky(p, Sigma, Lc) == 0) return 0;
  double tr = 0.0;
  for (int c = 0; c < p; ++c) tr += Sigma[c * p + c];
  double jit = 1e-10 * tr / p;
  for (int t = 1; t <= 12; ++t, jit *= 10.0) {
    for (int c = 0; c < p; ++c) Sigma[c * p + c] += jit;
    if (orc_cholesky(p, Sigma, Lc) == 0) return t;
  }
  return -1;
}

/* ------------------------------------------------------------------------------------------ */
/* Systematic resampling (Algorithm 2 step (e); the paper uses multinomial resampling, the        */
/* workloads here use systematic). Weights are quantised to integers w_i = floor(W_i * 2^40),      */
/* T = sum w_i, and position i is floor((i*T + floor(U*T)) / N); its ancestor is the first j      */
/* whose inclusive cumulative sum exceeds it. Exact integer arithmetic, no rounding order.        */
/* Requires N < 2^23 so that i*T fits in 64 bits.                                                  */
/* ------------------------------------------------------------------------------------------ */
void orc_resample(int N, const double *W, double U, int32_t *anc) {
  uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * N);
  uint64_t T = 0;
  for (int i = 0; i < N; ++i) {
    T += (uint64_t)floor(W[i] * 0x1.0p40);
    cum[i] = T;
  }
  if (T == 0) { /* no representable weight: keep every particle */
    for (int i = 0; i < N; ++i) anc[i] = i;
    free(cum);
    return;
  }
  uint64_t off = (uint64_t)floor(U * (double)T);
  int j = 0;
  for (int i = 0; i < N; ++i) {
    uint64_t pos = ((uint64_t)i * T + off) / (uint64_t)N;
    while (cum[j] <= pos) ++j;
    anc[i] = j;
  }
  free(cum);
}

/* ------------------------------------------------------------------------------------------ */
/* Multinomial resampling, the paper's scheme (Sec. 2.2): N independent draws from the weights.   */
/* On the same integer weights as above, offspring i takes position min(floor(U_i*T), T-1), with  */
/* its own uniform U_i, and its ancestor is the first j whose inclusive cumulative sum exceeds it */
/* (the inverse of the quantised CDF).                                                             */
/* ------------------------------------------------------------------------------------------ */
void orc_resample_multinomial(int N, const double *W, const double *U, int32_t *anc) {
  uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * N);
  uint64_t T = 0;
  for (int i = 0; i < N; ++i) {
    T += (uint64_t)floor(W[i] * 0x1.0p40);
    cum[i] = T;
  }
  for (int i = 0; i < N; ++i) {
    if (T == 0) {
      anc[i] = i;
      continue;
    }
    uint64_t pos = (uint64_t)floor(U[i] * (double)T);
    if (pos > T - 1) pos = T - 1;
    int j = 0;
    while (cum[j] <= pos) ++j;
    anc[i] = j;
  }
  free(cum);
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
