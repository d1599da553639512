// Stage-level kernels of subsampling SMC (Algorithm 2): data packing, control-variate moments
// (Sec. 3.2), the Newton step for the control-variate centre, particle initialisation, the
// temperature search and reweighting (Sec. 2.2, Sec. 3.3, Sec. 3.5), weighted moments and the mass
// matrix (Algorithm 2 (d)), and systematic resampling (Algorithm 2 (e)).
#include <cuda_bf16.h>
#include <math.h>

#include <type_traits>

#include "device.cuh"
#include "internal.h"

namespace subsmc {

namespace {

// Block-wide sum of one double (blockDim.x <= 1024). Result valid on every thread.
__device__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  for (int k = 0; k < nw; ++k) t += red[k];
  return t;
}

template <typename CT> __device__ __forceinline__ double ld_state(const void *p, int64_t i) {
  return (double)reinterpret_cast<const CT *>(p)[i];
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Packing: row k of Xp = [x_k | 0 .. | tail {c0, c1, c2, y_k} | 0 ..], stride S elements (a multiple
// of 64 bytes). The tail starts the 16-byte vector that follows the covariates (element Yo) and
// holds four values of the state type CT; its constants are written by k_row_consts once the
// control-variate centre is known and are zero until then.
// ------------------------------------------------------------------------------------------------
template <typename E, typename CT>
__global__ void k_pack(const E *X, int64_t n, int p, int64_t ld, const CT *y, E *Xp, int S,
                       int Yo) {
  constexpr int YS = sizeof(CT) / sizeof(E);  // elements per state-type value
  const int yo = Yo + 3 * YS;                 // y is the tail's fourth value
  const int64_t total = n * (int64_t)S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / S;
    const int s = (int)(t - k * S);
    E v;
    if (s >= yo && s < yo + YS) {
      const CT yk = y[k];
      v = reinterpret_cast<const E *>(&yk)[s - yo];
    } else if (s < p) {
      v = X[k * ld + s];
    } else {
      v = E(0);
    }
    Xp[t] = v;
  }
}

int pack_rows(const void *X, int x_dtype, int64_t n, int p, int64_t ld, const void *y, void *Xp,
              int S, int Yo, cudaStream_t s) {
  const int64_t total = n * (int64_t)S;
  const int grid = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
  if (x_dtype == 0)
    k_pack<uint64_t, double><<<grid, 256, 0, s>>>((const uint64_t *)X, n, p, ld,
                                                  (const double *)y, (uint64_t *)Xp, S, Yo);
  else if (x_dtype == 1)
    k_pack<uint32_t, float><<<grid, 256, 0, s>>>((const uint32_t *)X, n, p, ld, (const float *)y,
                                                (uint32_t *)Xp, S, Yo);
  else
    k_pack<uint16_t, float><<<grid, 256, 0, s>>>((const uint16_t *)X, n, p, ld, (const float *)y,
                                                (uint16_t *)Xp, S, Yo);
  return (int)cudaGetLastError();
}

// Per-row constants at the centre theta_bar (state type): one thread per row forms
// eta_bar = x'theta_bar in column order and rewrites c0..c2 of the row's tail (device.cuh).
template <typename XT, int FAM>
__global__ void k_row_consts(XT *Xp, int64_t n, int p, int S, int Yo,
                             const typename Store<XT>::CT *tb, typename Store<XT>::CT inv_s2,
                             typename Store<XT>::CT nu) {
  using SD = Store<XT>;
  using CT = typename SD::CT;
  const int nvx = Yo * (int)sizeof(XT) / 16;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    XT *row = Xp + k * S;
    CT eb = CT(0);
    for (int v = 0; v < nvx; ++v) {
      CT x[SD::VEC];
      SD::unpack(*reinterpret_cast<const uint4 *>(row + v * SD::VEC), x);
#pragma unroll
      for (int e = 0; e < SD::VEC; ++e) {
        const int c = v * SD::VEC + e;
        if (c < p) eb = fma(x[e], tb[c], eb);
      }
    }
    RowC<CT> *tl = reinterpret_cast<RowC<CT> *>(row + Yo);
    *tl = row_consts<FAM, CT>(eb, tl->y, inv_s2, nu);
  }
}

template <typename XT>
int launch_row_consts(XT *Xp, int64_t n, int p, int S, int Yo, int fam, const void *tb,
                      double inv_s2, double nu, cudaStream_t s) {
  using CT = typename Store<XT>::CT;
  const int64_t need = (n + 255) / 256;
  const int grid = (int)(need < 152 * 16 ? need : 152 * 16);
  const CT *t = (const CT *)tb;
  const CT i2 = (CT)inv_s2, v = (CT)nu;
  switch (fam) {
    case 0: k_row_consts<XT, 0><<<grid, 256, 0, s>>>(Xp, n, p, S, Yo, t, i2, v); break;
    case 1: k_row_consts<XT, 1><<<grid, 256, 0, s>>>(Xp, n, p, S, Yo, t, i2, v); break;
    case 2: k_row_consts<XT, 2><<<grid, 256, 0, s>>>(Xp, n, p, S, Yo, t, i2, v); break;
    case 3: k_row_consts<XT, 3><<<grid, 256, 0, s>>>(Xp, n, p, S, Yo, t, i2, v); break;
    default: k_row_consts<XT, 4><<<grid, 256, 0, s>>>(Xp, n, p, S, Yo, t, i2, v); break;
  }
  return (int)cudaGetLastError();
}

int row_consts(void *Xp, int x_dtype, int64_t n, int p, int S, int Yo, int fam, const void *tb_ct,
               double inv_s2, double nu, cudaStream_t s) {
  if (n <= 0) return 0;
  if (x_dtype == 0)
    return launch_row_consts<double>((double *)Xp, n, p, S, Yo, fam, tb_ct, inv_s2, nu, s);
  if (x_dtype == 1)
    return launch_row_consts<float>((float *)Xp, n, p, S, Yo, fam, tb_ct, inv_s2, nu, s);
  return launch_row_consts<__nv_bfloat16>((__nv_bfloat16 *)Xp, n, p, S, Yo, fam, tb_ct, inv_s2, nu,
                                          s);
}

// ------------------------------------------------------------------------------------------------
// Control-variate moments at theta (Sec. 3.2): A = sum_k l_k, B = sum_k l'_k x_k,
// C = sum_k l''_k x_k x_k'. Rows go through shared memory in tiles of 32: one lane per row forms
// eta_bar in FP64 and evaluates the family terms in FP64; the tile's contributions to C are
// accumulated in AT (FP64 for FP64 storage, FP32 otherwise: products of stored FP32/BF16 values) and
// added to per-thread FP64 accumulators once per tile; A and B stay FP64 throughout. Each thread
// owns fixed (r, c) pairs of the upper triangle; block partials are summed in block order.
// ------------------------------------------------------------------------------------------------
constexpr int kCvThreads = 256, kCvTile = 32, kCvMaxPairs = 32;

template <typename XT>
__device__ __forceinline__ double packed_x(const XT *row, int slot);
template <> __device__ __forceinline__ double packed_x<double>(const double *row, int slot) {
  return row[slot];
}
template <> __device__ __forceinline__ double packed_x<float>(const float *row, int slot) {
  return (double)row[slot];
}
template <>
__device__ __forceinline__ double packed_x<__nv_bfloat16>(const __nv_bfloat16 *row, int slot) {
  return (double)__bfloat162float(row[slot]);
}
template <typename XT> __device__ __forceinline__ double packed_y(const XT *row, int Yo) {
  return (double)reinterpret_cast<const RowC<typename Store<XT>::CT> *>(row + Yo)->y;
}

template <typename XT, int MAXQ>
__global__ void __launch_bounds__(kCvThreads) k_cv_partials(const XT *Xp, int64_t n, int p, int S,
                                                            int Yo, int fam, double s2,
                                                            double nu, const double *theta,
                                                            double *part) {
  using AT = typename std::conditional<sizeof(XT) == 8, double, float>::type;
  extern __shared__ double sh[];
  double *ths = sh;                                   // [p]
  double *d1s = ths + p;                              // [kCvTile]
  double *red = d1s + kCvTile;                        // [32]
  AT *xs = reinterpret_cast<AT *>(red + 32);          // [kCvTile][p]
  AT *wx = xs + kCvTile * p;                          // [kCvTile][p]   l'' * x
  AT *d2s = wx + kCvTile * p;                         // [kCvTile]
  const int tid = threadIdx.x;
  const int np = p * (p + 1) / 2;
  for (int c = tid; c < p; c += blockDim.x) ths[c] = theta[c];
  int qr[MAXQ], qc[MAXQ];
  double acc[MAXQ];
#pragma unroll
  for (int i = 0; i < MAXQ; ++i) {
    const int q = tid + i * kCvThreads;
    int r = 0, c = 0;
    if (q < np) {  // row-major enumeration of the upper triangle
      int rem = q;
      while (rem >= p - r) {
        rem -= p - r;
        ++r;
      }
      c = r + rem;
    }
    qr[i] = r;
    qc[i] = c;
    acc[i] = 0.0;
  }
  double Bacc = 0.0, Aacc = 0.0;
  __syncthreads();
  const int64_t ntiles = (n + kCvTile - 1) / kCvTile;
  for (int64_t tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    const int64_t k0 = tile * kCvTile;
    // stage the tile's covariates (row-major over the tile)
    for (int e = tid; e < kCvTile * p; e += blockDim.x) {
      const int rr = e / p, c = e - rr * p;
      const int64_t k = k0 + rr;
      xs[e] = k < n ? (AT)packed_x<XT>(Xp + k * S, c) : AT(0);
    }
    __syncthreads();
    // one lane per row: eta_bar and the family terms in FP64
    if (tid < kCvTile) {
      const int64_t k = k0 + tid;
      double l = 0.0, d1 = 0.0, d2 = 0.0;
      if (k < n) {
        double eta = 0.0;
        for (int c = 0; c < p; ++c) eta = fma((double)xs[tid * p + c], ths[c], eta);
        const double y = packed_y<XT>(Xp + k * S, Yo);
        switch (fam) {
          case 0: row_value<0>(eta, y, s2, nu, l, d1, d2); break;
          case 1: row_value<1>(eta, y, s2, nu, l, d1, d2); break;
          case 2: row_value<2>(eta, y, s2, nu, l, d1, d2); break;
          case 3: row_value<3>(eta, y, s2, nu, l, d1, d2); break;
          default: row_value<4>(eta, y, s2, nu, l, d1, d2); break;
        }
      }
      d1s[tid] = d1;
      d2s[tid] = (AT)d2;
      Aacc += l;
    }
    __syncthreads();
    for (int e = tid; e < kCvTile * p; e += blockDim.x) wx[e] = d2s[e / p] * xs[e];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < MAXQ; ++i) {
      if (tid + i * kCvThreads < np) {
        AT t = AT(0);
#pragma unroll 8
        for (int rr = 0; rr < kCvTile; ++rr) t = fma(wx[rr * p + qr[i]], xs[rr * p + qc[i]], t);
        acc[i] += (double)t;
      }
    }
    if (tid < p)
      for (int rr = 0; rr < kCvTile; ++rr) Bacc = fma(d1s[rr], (double)xs[rr * p + tid], Bacc);
    __syncthreads();
  }
  double *out = part + (int64_t)blockIdx.x * (1 + p + np);
  const double A = block_sum(Aacc, red);
  if (tid == 0) out[0] = A;
  if (tid < p) out[1 + tid] = Bacc;
#pragma unroll
  for (int i = 0; i < MAXQ; ++i) {
    const int q = tid + i * kCvThreads;
    if (q < np) out[1 + p + q] = acc[i];
  }
}

__global__ void k_cv_reduce(const double *part, int nblk, int p, double *A, double *B, double *C) {
  const int np = p * (p + 1) / 2, width = 1 + p + np;
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; e < width; e += warps) {
    double s = 0.0;  // lanes over blocks, then a fixed warp tree: deterministic
    for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * width + e];
    s = warp_sum(s);
    if (lane != 0) continue;
    if (e == 0) {
      *A = s;
    } else if (e <= p) {
      B[e - 1] = s;
    } else {
      int rem = e - 1 - p, r = 0;
      while (rem >= p - r) {
        rem -= p - r;
        ++r;
      }
      const int c = r + rem;
      C[r * p + c] = s;
      C[c * p + r] = s;
    }
  }
}

template <typename XT, int MAXQ>
cudaError_t launch_cv_q(int nblocks, size_t smem, cudaStream_t s, const XT *Xp, int64_t n, int p,
                        int S, int Yo, int fam, double s2, double nu, const double *theta,
                        double *part) {
  cudaError_t e = cudaFuncSetAttribute(k_cv_partials<XT, MAXQ>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_cv_partials<XT, MAXQ><<<nblocks, kCvThreads, smem, s>>>(Xp, n, p, S, Yo, fam, s2, nu,
                                                            theta, part);
  return cudaGetLastError();
}

// Pair slots per thread: the smallest compiled count that covers p(p+1)/2 pairs.
template <typename XT>
cudaError_t launch_cv(int need, int nblocks, size_t smem, cudaStream_t s, const XT *Xp, int64_t n,
                      int p, int S, int Yo, int fam, double s2, double nu, const double *theta,
                      double *part) {
  if (need <= 1) return launch_cv_q<XT, 1>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
  if (need <= 2) return launch_cv_q<XT, 2>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
  if (need <= 4) return launch_cv_q<XT, 4>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
  if (need <= 8) return launch_cv_q<XT, 8>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
  if (need <= 16) return launch_cv_q<XT, 16>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
  return launch_cv_q<XT, 32>(nblocks, smem, s, Xp, n, p, S, Yo, fam, s2, nu, theta, part);
}

int cv_moments_blocks(int p) {
  (void)p;
  return 2 * 152;
}

int cv_moments(const void *Xp, int x_dtype, int64_t n, int p, int S, int Yo, int fam, double sigma2,
               double nu, const double *theta, double *partials, int nblocks, double *A, double *B,
               double *C, int mode, cudaStream_t s) {
  if (mode == 0 && x_dtype == 2 && p <= 128) {
    int used = 0;
    const int e =
        cv_moments_mma(Xp, n, p, S, Yo, fam, sigma2, nu, theta, partials, nblocks, &used, s);
    if (e != 0) return e;
    const int width = 1 + p + p * (p + 1) / 2;
    k_cv_reduce<<<(width + 7) / 8, 256, 0, s>>>(partials, used, p, A, B, C);
    return (int)cudaGetLastError();
  }
  if (p * (p + 1) / 2 > kCvThreads * kCvMaxPairs) return (int)cudaErrorInvalidValue;
  const size_t at = x_dtype == 0 ? sizeof(double) : sizeof(float);
  const size_t smem = (size_t)(p + kCvTile + 32) * sizeof(double) + (2 * kCvTile * p + kCvTile) * at;
  const int np = p * (p + 1) / 2, need = (np + kCvThreads - 1) / kCvThreads;
  cudaError_t e;
  if (x_dtype == 0)
    e = launch_cv<double>(need, nblocks, smem, s, (const double *)Xp, n, p, S, Yo, fam, sigma2,
                          nu, theta, partials);
  else if (x_dtype == 1)
    e = launch_cv<float>(need, nblocks, smem, s, (const float *)Xp, n, p, S, Yo, fam, sigma2, nu,
                         theta, partials);
  else
    e = launch_cv<__nv_bfloat16>(need, nblocks, smem, s, (const __nv_bfloat16 *)Xp, n, p, S, Yo,
                                 fam, sigma2, nu, theta, partials);
  if (e != cudaSuccess) return (int)e;
  const int width = 1 + p + p * (p + 1) / 2;
  k_cv_reduce<<<(width + 7) / 8, 256, 0, s>>>(partials, nblocks, p, A, B, C);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Dense FP64 Cholesky of a p x p SPD matrix held in shared memory by one block (right-looking).
// Returns false (on every thread) if a pivot is not positive.
// ------------------------------------------------------------------------------------------------
__device__ bool chol_block(double *M, int p, int *flag) {
  const int tid = threadIdx.x, bs = blockDim.x;
  if (tid == 0) *flag = 0;
  __syncthreads();
  for (int j = 0; j < p; ++j) {
    if (tid == 0) {
      const double v = M[j * p + j];
      if (!(v > 0.0) || !isfinite(v))
        *flag = 1;
      else
        M[j * p + j] = sqrt(v);
    }
    __syncthreads();
    if (*flag) return false;
    const double piv = M[j * p + j];
    for (int i = j + 1 + tid; i < p; i += bs) M[i * p + j] /= piv;
    __syncthreads();
    const int w = p - j - 1;
    for (int e = tid; e < w * w; e += bs) {
      const int i = j + 1 + e / w, k = j + 1 + e % w;
      if (k <= i) M[i * p + k] -= M[i * p + j] * M[k * p + j];
    }
    __syncthreads();
  }
  for (int e = tid; e < p * p; e += bs) {  // zero the strict upper triangle
    const int i = e / p, k = e % p;
    if (k > i) M[e] = 0.0;
  }
  __syncthreads();
  return true;
}

// Newton step for the posterior mode: solve (-C + diag(1/v)) step = B - (theta - mu)/v.
__global__ void k_newton_step(int p, const double *theta, const double *B, const double *C,
                              const double *mu, const double *var, double *step, int *info) {
  extern __shared__ double M[];
  __shared__ int flag;
  double *g = M + p * p;
  const int tid = threadIdx.x;
  for (int c = tid; c < p; c += blockDim.x) g[c] = B[c] - (theta[c] - mu[c]) / var[c];
  // M = -C + diag(1/var) + lam I. A log-density that is not concave (Student-t far from the mode)
  // can leave M indefinite; lam = 1e-8 max|diag| (times 10 per retry) then keeps the step an
  // ascent direction (Levenberg's damping). Uniform across the block: every thread sees the same
  // factorisation outcome.
  double scale = 0.0;
  for (int i = 0; i < p; ++i) scale = fmax(scale, fabs(-C[i * p + i] + 1.0 / var[i]));
  if (!(scale > 0.0)) scale = 1e-300;
  double lam = 0.0;
  bool ok = false;
  for (int tries = 0; tries < 40 && !ok; ++tries) {
    for (int e = tid; e < p * p; e += blockDim.x) {
      const int i = e / p, k = e % p;
      M[e] = -C[e] + (i == k ? 1.0 / var[i] + lam : 0.0);
    }
    __syncthreads();
    ok = chol_block(M, p, &flag);
    lam = lam == 0.0 ? 1e-8 * scale : 10.0 * lam;
  }
  if (!ok) {
    if (tid == 0) *info = 1;
    return;
  }
  if (tid == 0) {  // forward then back substitution (p <= 126: one thread is enough)
    for (int i = 0; i < p; ++i) {
      double s = g[i];
      for (int k = 0; k < i; ++k) s -= M[i * p + k] * g[k];
      g[i] = s / M[i * p + i];
    }
    for (int i = p - 1; i >= 0; --i) {
      double s = g[i];
      for (int k = i + 1; k < p; ++k) s -= M[k * p + i] * g[k];
      g[i] = s / M[i * p + i];
    }
    *info = 0;
  }
  __syncthreads();
  for (int c = tid; c < p; c += blockDim.x) step[c] = g[c];
}

int newton_step(int p, const double *theta, const double *B, const double *C, const double *mu,
                const double *var, double *step, double *work, int *info, cudaStream_t s) {
  (void)work;
  const size_t smem = (size_t)(p * p + p) * sizeof(double);
  cudaError_t e =
      cudaFuncSetAttribute(k_newton_step, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  k_newton_step<<<1, 256, smem, s>>>(p, theta, B, C, mu, var, step, info);
  return (int)cudaGetLastError();
}

__global__ void k_axpy(int p, const double *x, double t, const double *sv, double *out) {
  for (int c = threadIdx.x; c < p; c += blockDim.x) out[c] = x[c] + t * sv[c];
}
int axpy_vec(int p, const double *x, double t, const double *sv, double *out, cudaStream_t st) {
  k_axpy<<<1, 128, 0, st>>>(p, x, t, sv, out);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Initialisation (Algorithm 2 step 1): theta_i ~ N(mu, diag v), u_ij ~ U{0..n-1}, W = 1/N.
// ------------------------------------------------------------------------------------------------
template <typename CT>
__global__ void k_init(int N, int p, int m, int64_t n, uint64_t seed, const double *mu,
                       const double *var, CT *theta, int32_t *u, double *logW, double *W) {
  const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = tid; t < (int64_t)N * p; t += stride) {
    const int i = (int)(t / p), c = (int)(t % p);
    const Stream st(seed, kInitTheta, 0u, (uint32_t)i);
    theta[t] = (CT)(mu[c] + sqrt(var[c]) * stream_normal(st, (uint32_t)c));
  }
  const int halves = (m + 1) / 2;
  for (int64_t t = tid; t < (int64_t)N * halves; t += stride) {
    const int i = (int)(t / halves), b = (int)(t % halves);
    const Stream st(seed, kInitU, 0u, (uint32_t)i);
    uint64_t r0, r1;
    st.pair((uint32_t)b, r0, r1);
    u[(int64_t)i * m + 2 * b] = (int32_t)draw_index(r0, (uint64_t)n);
    if (2 * b + 1 < m) u[(int64_t)i * m + 2 * b + 1] = (int32_t)draw_index(r1, (uint64_t)n);
  }
  for (int64_t t = tid; t < N; t += stride) {
    logW[t] = -log((double)N);
    W[t] = 1.0 / (double)N;
  }
}

int init_particles(int is_f64, int N, int p, int m, int64_t n, uint64_t seed, const double *mu,
                   const double *var, void *theta, int32_t *u, double *logW, double *W,
                   cudaStream_t s) {
  const int grid = 152 * 8;
  if (is_f64)
    k_init<double><<<grid, 256, 0, s>>>(N, p, m, n, seed, mu, var, (double *)theta, u, logW, W);
  else
    k_init<float><<<grid, 256, 0, s>>>(N, p, m, n, seed, mu, var, (float *)theta, u, logW, W);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Temperature search and reweighting (Sec. 2.2, Sec. 3.3, Algorithm 2 (b)-(c)).
//   lw_i(D) = log W_i + D l_hat_i - ((a + D)^2 - a^2)/2 sigma2_hat_i,  ESS(D) = s1^2 / s2
// with s1 = sum e^{lw - M}, s2 = sum e^{2(lw - M)}, M = max lw (the exact FP64 maximum: early in
// the run |lw| reaches ~1e11, where a float maximum can miss the true one by ~1e4 and overflow
// exp). Round 0 also tests D = 1 - a; each round evaluates the K-1 interior points of the bracket
// and keeps the first sub-interval whose right end has ESS < tau N. Two launches per round (the
// maxima, then the sums); in each, a thread covers one candidate over a stream of particles, the
// block merges its streams, and the last block to finish merges the blocks' partials: thread
// (q, k) a fixed subset q of the blocks for candidate k (loads in flight together), then the
// subsets in order. Merges are maxima and FP64 sums only (an FP64 exponential costs about 1000
// cycles of a warp's issue on GB300, so none is spent outside the per-particle terms).
// ------------------------------------------------------------------------------------------------
constexpr int kMaxK = kSearchMaxK, kRwMaxBlocks = 152;
constexpr int kSwThreads = 128;   // search: threads per block (candidates x particle streams)
constexpr int kFinThreads = 128;  // final reweighting: threads per block

// Candidates of a search round. Bracket search (S = 0): round 0 evaluates the K - 1 interior
// points of [0, 1 - a] and the end point 1 - a itself (the test "ESS(1 - a) >= tau N" of the
// rule); later rounds evaluate the K - 1 interior points lo + (hi - lo) k / K of the current
// bracket. Grid (S > 0): round r evaluates grid points rK .. rK + K - 1 (ascending).
__device__ __forceinline__ int candidates(const DevState *st, int K, int round, int S,
                                          double &lo, double &hi) {
  if (S > 0) {
    lo = hi = st->dmax;
    return min(K, S - round * K);
  }
  lo = round == 0 ? 0.0 : st->lo;
  hi = round == 0 ? st->dmax : st->hi;
  return round == 0 ? K : K - 1;
}
__device__ __forceinline__ double candidate(double lo, double hi, int K, int k) {
  return k == K - 1 ? hi : lo + (hi - lo) * (k + 1) / K;
}
// Grid point s of S: (1 - a) 10^(-E (S - 1 - s) / (S - 1)); the last point is 1 - a exactly.
__device__ __forceinline__ double grid_point(double dmax, int S, double E, int s) {
  if (s >= S - 1) return dmax;
  return dmax * pow(10.0, -E * (double)(S - 1 - s) / (double)(S - 1));
}

// Per-block table of the round's candidates: D_k and h_k = ((a + D_k)^2 - a^2) / 2, so that
// lw_i(D_k) = log W_i + D_k l_hat_i - h_k sigma2_hat_i.
__device__ __forceinline__ int load_candidates(const DevState *st, int K, int round, int S,
                                               double E, double *Dk, double *hk, double &lo,
                                               double &hi) {
  const int ncand = candidates(st, K, round, S, lo, hi);
  const double a = st->a;
  for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
    const double D = S > 0 ? grid_point(st->dmax, S, E, round * K + k) : candidate(lo, hi, K, k);
    Dk[k] = D;
    hk[k] = 0.5 * ((a + D) * (a + D) - a * a);
  }
  return ncand;
}

// Lane layout of the search kernels: kslots = 16 lanes per candidate row when the round has at
// most 16 candidates (so a warp carries two particle streams and no lane idles), else 32.
struct SearchLanes {
  int kslots, nstream, k, stream;
  __device__ __forceinline__ explicit SearchLanes(int ncand) {
    kslots = ncand <= 16 ? 16 : 32;
    nstream = kSwThreads / kslots;
    k = (int)threadIdx.x % kslots;
    stream = (int)threadIdx.x / kslots;
  }
};

// Signals the block that finishes last (ticket in the device state). Call after the block's
// partials are written; every thread receives the answer. nblk: the problem's blocks.
__device__ __forceinline__ bool last_block(DevState *st, bool *flag, int nblk) {
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) *flag = atomicAdd(&st->ticket, 1u) == (unsigned)nblk - 1;
  __syncthreads();
  if (*flag) __threadfence();
  return *flag;
}

// Phase 1 of a round: max_i lw_i(D_k) per candidate.
__device__ __forceinline__ void k_search_max_body(int N, const double *ell, const double *sig2,
    const double *logW, int K, int round, int S, double E, DevState *st, double *pmax, double *gmax,
    int bid_, int nblk_) {
  __shared__ double Dk[kMaxK], hk[kMaxK];
  __shared__ double ws[kSwThreads];
  __shared__ bool is_last;
  if (st->search_done) return;  // uniform across the grid
  double lo, hi;
  const int ncand = load_candidates(st, K, round, S, E, Dk, hk, lo, hi);
  __syncthreads();
  const SearchLanes L(ncand);
  const int chunk = (N + nblk_ - 1) / nblk_;
  const int i0 = bid_ * chunk, i1 = min(N, i0 + chunk);
  double mx = -INFINITY;
  if (L.k < ncand) {
    const double D = Dk[L.k], h = hk[L.k];
#pragma unroll 4
    for (int i = i0 + L.stream; i < i1; i += L.nstream)
      mx = fmax(mx, fma(-h, sig2[i], fma(D, ell[i], logW[i])));
  }
  ws[threadIdx.x] = mx;
  __syncthreads();
  if ((int)threadIdx.x < ncand) {
    double m = ws[threadIdx.x];
    for (int q = 1; q < L.nstream; ++q) m = fmax(m, ws[q * L.kslots + threadIdx.x]);
    pmax[bid_ * kMaxK + threadIdx.x] = m;
  }
  if (!last_block(st, &is_last, nblk_)) return;
  double m = -INFINITY;
  if (L.k < ncand) {
#pragma unroll 8
    for (int b = L.stream; b < (int)nblk_; b += L.nstream)
      m = fmax(m, __ldcg(pmax + b * kMaxK + L.k));
  }
  ws[threadIdx.x] = m;
  __syncthreads();
  if ((int)threadIdx.x < ncand) {
    double g = ws[threadIdx.x];
    for (int q = 1; q < L.nstream; ++q) g = fmax(g, ws[q * L.kslots + threadIdx.x]);
    gmax[threadIdx.x] = g;
  }
  if (threadIdx.x == 0) st->ticket = 0;
}
__global__ void __launch_bounds__(kSwThreads)
    k_search_max(int N, const double *ell, const double *sig2, const double *logW, int K,
                 int round, int S, double E, DevState *st, double *pmax, double *gmax) {
  k_search_max_body(N, ell, sig2, logW, K, round, S, E, st, pmax, gmax, blockIdx.x, gridDim.x);
}

// Phase 2: s1 = sum e^{lw - M}, s2 = sum e^{2(lw - M)} (one exponential per particle and
// candidate), ESS = s1^2 / s2; the last block sums the block partials and updates the bracket:
// the first sub-interval whose right end has ESS < tau N.
__device__ __forceinline__ void k_search_sum_body(int N, const double *ell, const double *sig2,
    const double *logW, double tau, int K, int round, int last_round, int S, double E, DevState *st,
    const double *gmax, double *psum, int bid_, int nblk_) {
  __shared__ double Dk[kMaxK], hk[kMaxK], ess_k[kMaxK];
  __shared__ double w1[kSwThreads], w2[kSwThreads];
  __shared__ bool is_last;
  if (st->search_done) return;
  double lo, hi;
  const int ncand = load_candidates(st, K, round, S, E, Dk, hk, lo, hi);
  __syncthreads();
  const SearchLanes L(ncand);
  const int chunk = (N + nblk_ - 1) / nblk_;
  const int i0 = bid_ * chunk, i1 = min(N, i0 + chunk);
  double s1 = 0.0, s2 = 0.0;
  if (L.k < ncand) {
    const double D = Dk[L.k], h = hk[L.k], M = __ldcg(gmax + L.k);
    if (M > -INFINITY) {
#pragma unroll 4
      for (int i = i0 + L.stream; i < i1; i += L.nstream) {
        const double e = exp(fma(-h, sig2[i], fma(D, ell[i], logW[i])) - M);
        s1 += e;
        s2 = fma(e, e, s2);
      }
    }
  }
  w1[threadIdx.x] = s1;
  w2[threadIdx.x] = s2;
  __syncthreads();
  if ((int)threadIdx.x < ncand) {  // the streams of candidate k in stream order
    double t1 = w1[threadIdx.x], t2 = w2[threadIdx.x];
    for (int q = 1; q < L.nstream; ++q) {
      t1 += w1[q * L.kslots + threadIdx.x];
      t2 += w2[q * L.kslots + threadIdx.x];
    }
    psum[2 * (bid_ * kMaxK + threadIdx.x)] = t1;
    psum[2 * (bid_ * kMaxK + threadIdx.x) + 1] = t2;
  }
  if (!last_block(st, &is_last, nblk_)) return;
  {
    double t1 = 0.0, t2 = 0.0;
    if (L.k < ncand) {
#pragma unroll 8
      for (int b = L.stream; b < (int)nblk_; b += L.nstream) {
        t1 += __ldcg(psum + 2 * (b * kMaxK + L.k));
        t2 += __ldcg(psum + 2 * (b * kMaxK + L.k) + 1);
      }
    }
    w1[threadIdx.x] = t1;
    w2[threadIdx.x] = t2;
  }
  __syncthreads();
  if ((int)threadIdx.x < ncand) {
    double t1 = w1[threadIdx.x], t2 = w2[threadIdx.x];
    for (int q = 1; q < L.nstream; ++q) {
      t1 += w1[q * L.kslots + threadIdx.x];
      t2 += w2[q * L.kslots + threadIdx.x];
    }
    ess_k[threadIdx.x] = t1 * t1 / t2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double target = tau * (double)N;
  const int ninner = round == 0 ? K - 1 : ncand;  // interior points (round 0 adds the end point)
  for (int k = 0; k < ncand; ++k)
    if (!(ess_k[k] == ess_k[k])) atomicOr(&st->err, kErrNonFinite);
  if (S > 0) {  // grid rule: the closest ESS so far wins; ties keep the smaller increment
    for (int k = 0; k < ncand; ++k) {
      const double dist = fabs(ess_k[k] - target);
      if (dist < st->best_dist) {
        st->best_dist = dist;
        st->best_D = Dk[k];
      }
    }
    if (round == last_round) {
      st->D = st->best_D;
      st->search_done = 1;
    }
    st->ticket = 0;
    return;
  }
  if (round == 0 && ess_k[K - 1] >= target) {  // ESS(1 - a) >= target: go straight to a = 1
    st->D = st->dmax;
    st->search_done = 1;
    st->ticket = 0;
    return;
  }
  int first = ninner + 1;  // 1-based index of the first interior candidate with ESS < target
  for (int k = 0; k < ninner; ++k) {
    if (ess_k[k] < target) {
      first = k + 1;
      break;
    }
  }
  const double nlo = lo + (hi - lo) * (first - 1) / K;
  const double nhi = first <= ninner ? lo + (hi - lo) * first / K : hi;
  st->lo = nlo;
  st->hi = nhi;
  if (round == last_round) {
    st->D = nlo > 0.0 ? nlo : nhi;
    st->search_done = 1;
  }
  st->ticket = 0;
}
__global__ void __launch_bounds__(kSwThreads)
    k_search_sum(int N, const double *ell, const double *sig2, const double *logW, double tau,
                 int K, int round, int last_round, int S, double E, DevState *st,
                 const double *gmax, double *psum) {
  k_search_sum_body(N, ell, sig2, logW, tau, K, round, last_round, S, E, st, gmax, psum, blockIdx.x,
      gridDim.x);
}

// Final reweighting: log-sum-exps of the new (x = lw(D)) and old (x = log W) log weights, the
// ESS at D and the log Z increment (Sec. 3.5). Same two phases; index 0 = new, 1 = old. Within a
// block the threads' values are combined by a fixed tree; the last block combines the blocks'
// partials in the same way (thread t the blocks t, t + 128, ..).
__device__ __forceinline__ void tree_max2(double *v0, double *v1) {
  for (int w = kFinThreads / 2; w > 0; w >>= 1) {
    __syncthreads();
    if ((int)threadIdx.x < w) {
      v0[threadIdx.x] = fmax(v0[threadIdx.x], v0[threadIdx.x + w]);
      v1[threadIdx.x] = fmax(v1[threadIdx.x], v1[threadIdx.x + w]);
    }
  }
  __syncthreads();
}
__device__ __forceinline__ void tree_sum3(double *v0, double *v1, double *v2) {
  for (int w = kFinThreads / 2; w > 0; w >>= 1) {
    __syncthreads();
    if ((int)threadIdx.x < w) {
      v0[threadIdx.x] += v0[threadIdx.x + w];
      v1[threadIdx.x] += v1[threadIdx.x + w];
      v2[threadIdx.x] += v2[threadIdx.x + w];
    }
  }
  __syncthreads();
}

__device__ __forceinline__ void k_final_max_body(int N, const double *ell, const double *sig2,
    const double *logW, DevState *st, double *pmax, double *gmax, int bid_, int nblk_) {
  __shared__ double v0[kFinThreads], v1[kFinThreads];
  __shared__ bool is_last;
  const double a = st->a, D = st->D, h = 0.5 * ((a + D) * (a + D) - a * a);
  const int tid = threadIdx.x, stride = nblk_ * blockDim.x;
  double m0 = -INFINITY, m1 = -INFINITY;
  for (int i = bid_ * blockDim.x + tid; i < N; i += stride) {
    const double lw = logW[i];
    m0 = fmax(m0, fma(-h, sig2[i], fma(D, ell[i], lw)));
    m1 = fmax(m1, lw);
  }
  v0[tid] = m0;
  v1[tid] = m1;
  tree_max2(v0, v1);
  if (tid == 0) {
    pmax[2 * bid_] = v0[0];
    pmax[2 * bid_ + 1] = v1[0];
  }
  if (!last_block(st, &is_last, nblk_)) return;
  m0 = m1 = -INFINITY;
  for (int b = tid; b < (int)nblk_; b += blockDim.x) {
    m0 = fmax(m0, __ldcg(pmax + 2 * b));
    m1 = fmax(m1, __ldcg(pmax + 2 * b + 1));
  }
  v0[tid] = m0;
  v1[tid] = m1;
  tree_max2(v0, v1);
  if (tid == 0) {
    gmax[0] = v0[0];
    gmax[1] = v1[0];
    st->ticket = 0;
  }
}
__global__ void __launch_bounds__(kFinThreads)
    k_final_max(int N, const double *ell, const double *sig2, const double *logW, DevState *st,
                double *pmax, double *gmax) {
  k_final_max_body(N, ell, sig2, logW, st, pmax, gmax, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void k_final_sum_body(int N, const double *ell, const double *sig2,
    const double *logW, DevState *st, const double *gmax, double *psum, int bid_, int nblk_) {
  __shared__ double v0[kFinThreads], v1[kFinThreads], v2[kFinThreads];
  __shared__ bool is_last;
  const double a = st->a, D = st->D, h = 0.5 * ((a + D) * (a + D) - a * a);
  const double M0 = __ldcg(gmax), M1 = __ldcg(gmax + 1);
  const int tid = threadIdx.x, stride = nblk_ * blockDim.x;
  double s1 = 0.0, s2 = 0.0, so = 0.0;
  for (int i = bid_ * blockDim.x + tid; i < N; i += stride) {
    const double lw = logW[i];
    const double e = exp(fma(-h, sig2[i], fma(D, ell[i], lw)) - M0);
    s1 += e;
    s2 = fma(e, e, s2);
    so += exp(lw - M1);
  }
  v0[tid] = s1;
  v1[tid] = s2;
  v2[tid] = so;
  tree_sum3(v0, v1, v2);
  if (tid == 0) {
    psum[3 * bid_] = v0[0];
    psum[3 * bid_ + 1] = v1[0];
    psum[3 * bid_ + 2] = v2[0];
  }
  if (!last_block(st, &is_last, nblk_)) return;
  s1 = s2 = so = 0.0;
  for (int b = tid; b < (int)nblk_; b += blockDim.x) {
    s1 += __ldcg(psum + 3 * b);
    s2 += __ldcg(psum + 3 * b + 1);
    so += __ldcg(psum + 3 * b + 2);
  }
  v0[tid] = s1;
  v1[tid] = s2;
  v2[tid] = so;
  tree_sum3(v0, v1, v2);
  if (tid != 0) return;
  const double lse_new = M0 + log(v0[0]), lse_old = M1 + log(v2[0]);
  st->lse_new = lse_new;
  st->lse_old = lse_old;
  st->ess = v0[0] * v0[0] / v1[0];
  st->log_z_inc = lse_new - lse_old;
  st->log_z += st->log_z_inc;
  st->a_prev = a;
  st->a = (D == st->dmax) ? 1.0 : a + D;
  if (!isfinite(lse_new) || !isfinite(lse_old)) atomicOr(&st->err, kErrNonFinite);
  st->ticket = 0;
}
__global__ void __launch_bounds__(kFinThreads)
    k_final_sum(int N, const double *ell, const double *sig2, const double *logW, DevState *st,
                const double *gmax, double *psum) {
  k_final_sum_body(N, ell, sig2, logW, st, gmax, psum, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void k_normalise_body(int N, const double *ell, const double *sig2,
    double *logW, double *W, const DevState *st, int bid_, int nblk_) {
  const double a = st->a_prev, D = st->D, lse = st->lse_new;
  const double h = 0.5 * ((a + D) * (a + D) - a * a);
  for (int i = bid_ * blockDim.x + threadIdx.x; i < N; i += nblk_ * blockDim.x) {
    const double l = fma(-h, sig2[i], fma(D, ell[i], logW[i])) - lse;
    logW[i] = l;
    W[i] = exp(l);
  }
}
__global__ void k_normalise(int N, const double *ell, const double *sig2, double *logW, double *W,
                            const DevState *st) {
  k_normalise_body(N, ell, sig2, logW, W, st, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void k_search_begin_body(DevState *st, int bid_, int nblk_) {
  st->dmax = 1.0 - st->a;
  st->lo = 0.0;
  st->hi = st->dmax;
  st->D = 0.0;
  st->best_dist = INFINITY;
  st->best_D = st->dmax;
  st->search_done = 0;
  st->ticket = 0;
}
__global__ void k_search_begin(DevState *st) {
  k_search_begin_body(st, blockIdx.x, gridDim.x);
}

// ------------------------------------------------------------------------------------------------
// The whole reweighting of one problem in one launch: the search rounds and the final log-sum-exps
// above, separated by grid barriers instead of kernel boundaries. Every phase keeps the block count
// and the per-block work of its separate launch, and every block repeats the merge that the last
// block does there (same loads, same order), so the results are those of the separate launches bit
// for bit; block 0 alone writes the device state.
// ------------------------------------------------------------------------------------------------
constexpr long long kBarrierCycles = 4000000000ll;  // about 2 s at the maximum SM clock

// Grid-wide barrier of a launch whose blocks are all resident at once (at most one small block per
// SM, launched alone in its stream): arrivals counted in st->ticket, release by advancing
// st->ticket2. Bounded: a block that waits about 2 s, or that finds another block has given up,
// sets kErrCap and returns false on every thread (the kernel then leaves).
__device__ __forceinline__ bool grid_barrier(DevState *st, int nblk, int *flag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int *gen = &st->ticket2;
    volatile int *err = &st->err;
    const unsigned int g0 = *gen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(&st->ticket, 1u) == (unsigned)nblk - 1) {
      atomicExch(&st->ticket, 0u);
      __threadfence();
      atomicAdd(&st->ticket2, 1u);
    } else {
      const long long t0 = clock64();
      while (*gen == g0) {
        if ((*err & kErrCap) || clock64() - t0 > kBarrierCycles) {
          ok = 0;
          break;
        }
      }
    }
    if (!ok) atomicOr(&st->err, kErrCap);
    __threadfence();
    *flag = ok;
  }
  __syncthreads();
  return *flag != 0;
}

// The search bracket of one stage, kept by every block of the one-launch reweighting.
struct SearchState {
  double a, dmax, lo, hi, D, best_dist, best_D;
  int done;
};

__device__ __forceinline__ int state_candidates(const SearchState &ss, int K, int round, int S,
                                                double E, double *Dk, double *hk, double &lo,
                                                double &hi) {
  int ncand;
  if (S > 0) {
    lo = hi = ss.dmax;
    ncand = min(K, S - round * K);
  } else {
    lo = round == 0 ? 0.0 : ss.lo;
    hi = round == 0 ? ss.dmax : ss.hi;
    ncand = round == 0 ? K : K - 1;
  }
  const double a = ss.a;
  for (int k = threadIdx.x; k < ncand; k += blockDim.x) {
    const double D = S > 0 ? grid_point(ss.dmax, S, E, round * K + k) : candidate(lo, hi, K, k);
    Dk[k] = D;
    hk[k] = 0.5 * ((a + D) * (a + D) - a * a);
  }
  return ncand;
}

// nbs: the blocks of a search round, nb: the blocks of the final reweighting (gridDim.x is the
// larger); part: the same scratch as the separate launches.
__global__ void __launch_bounds__(kSwThreads)
    k_reweight_one(int N, const double *ell, const double *sig2, double *logW, double *W,
                   double tau, int K, int rounds, int S, double E, DevState *st, double *part,
                   int nbs, int nb) {
  __shared__ double Dk[kMaxK], hk[kMaxK], ess_k[kMaxK], gm[kMaxK];
  __shared__ double w1[kSwThreads], w2[kSwThreads], w3[kSwThreads];
  __shared__ SearchState ss;
  __shared__ int flag;
  const int bid = blockIdx.x, tid = threadIdx.x, nblk = gridDim.x;
  double *pmax = part + kMaxK, *psum = pmax + kRwMaxBlocks * kMaxK;
  if (tid == 0) {
    ss.a = st->a;
    ss.dmax = 1.0 - ss.a;
    ss.lo = 0.0;
    ss.hi = ss.dmax;
    ss.D = 0.0;
    ss.best_dist = INFINITY;
    ss.best_D = ss.dmax;
    ss.done = 0;
  }
  __syncthreads();
  const double target = tau * (double)N;
  for (int r = 0; r < rounds && !ss.done; ++r) {
    double lo, hi;
    const int ncand = state_candidates(ss, K, r, S, E, Dk, hk, lo, hi);
    __syncthreads();
    const SearchLanes L(ncand);
    const int chunk = (N + nbs - 1) / nbs;
    const int i0 = bid * chunk, i1 = min(N, i0 + chunk);
    if (bid < nbs) {  // the maxima of this block's particles (k_search_max)
      double mx = -INFINITY;
      if (L.k < ncand) {
        const double D = Dk[L.k], h = hk[L.k];
#pragma unroll 4
        for (int i = i0 + L.stream; i < i1; i += L.nstream)
          mx = fmax(mx, fma(-h, sig2[i], fma(D, ell[i], logW[i])));
      }
      w1[tid] = mx;
      __syncthreads();
      if (tid < ncand) {
        double m = w1[tid];
        for (int q = 1; q < L.nstream; ++q) m = fmax(m, w1[q * L.kslots + tid]);
        pmax[bid * kMaxK + tid] = m;
      }
    }
    if (!grid_barrier(st, nblk, &flag)) return;
    {  // every block: the maxima over blocks, merged as the last block of k_search_max does
      double m = -INFINITY;
      if (L.k < ncand) {
#pragma unroll 8
        for (int b = L.stream; b < nbs; b += L.nstream) m = fmax(m, __ldcg(pmax + b * kMaxK + L.k));
      }
      w1[tid] = m;
      __syncthreads();
      if (tid < ncand) {
        double g = w1[tid];
        for (int q = 1; q < L.nstream; ++q) g = fmax(g, w1[q * L.kslots + tid]);
        gm[tid] = g;
      }
      __syncthreads();
    }
    if (bid < nbs) {  // the sums of this block's particles (k_search_sum)
      double s1 = 0.0, s2 = 0.0;
      if (L.k < ncand) {
        const double D = Dk[L.k], h = hk[L.k], M = gm[L.k];
        if (M > -INFINITY) {
#pragma unroll 4
          for (int i = i0 + L.stream; i < i1; i += L.nstream) {
            const double e = exp(fma(-h, sig2[i], fma(D, ell[i], logW[i])) - M);
            s1 += e;
            s2 = fma(e, e, s2);
          }
        }
      }
      w1[tid] = s1;
      w2[tid] = s2;
      __syncthreads();
      if (tid < ncand) {
        double t1 = w1[tid], t2 = w2[tid];
        for (int q = 1; q < L.nstream; ++q) {
          t1 += w1[q * L.kslots + tid];
          t2 += w2[q * L.kslots + tid];
        }
        psum[2 * (bid * kMaxK + tid)] = t1;
        psum[2 * (bid * kMaxK + tid) + 1] = t2;
      }
    }
    if (!grid_barrier(st, nblk, &flag)) return;
    {  // every block: the ESS of each candidate, merged as the last block of k_search_sum does
      double t1 = 0.0, t2 = 0.0;
      if (L.k < ncand) {
#pragma unroll 8
        for (int b = L.stream; b < nbs; b += L.nstream) {
          t1 += __ldcg(psum + 2 * (b * kMaxK + L.k));
          t2 += __ldcg(psum + 2 * (b * kMaxK + L.k) + 1);
        }
      }
      w1[tid] = t1;
      w2[tid] = t2;
      __syncthreads();
      if (tid < ncand) {
        t1 = w1[tid];
        t2 = w2[tid];
        for (int q = 1; q < L.nstream; ++q) {
          t1 += w1[q * L.kslots + tid];
          t2 += w2[q * L.kslots + tid];
        }
        ess_k[tid] = t1 * t1 / t2;
      }
      __syncthreads();
    }
    if (tid == 0) {  // the bracket (the same arithmetic in every block)
      const int ninner = r == 0 ? K - 1 : ncand;
      if (bid == 0)
        for (int k = 0; k < ncand; ++k)
          if (!(ess_k[k] == ess_k[k])) atomicOr(&st->err, kErrNonFinite);
      if (S > 0) {  // grid rule: the closest ESS so far wins; ties keep the smaller increment
        for (int k = 0; k < ncand; ++k) {
          const double dist = fabs(ess_k[k] - target);
          if (dist < ss.best_dist) {
            ss.best_dist = dist;
            ss.best_D = Dk[k];
          }
        }
        if (r == rounds - 1) {
          ss.D = ss.best_D;
          ss.done = 1;
        }
      } else if (r == 0 && ess_k[K - 1] >= target) {  // go straight to a = 1
        ss.D = ss.dmax;
        ss.done = 1;
      } else {
        int first = ninner + 1;
        for (int k = 0; k < ninner; ++k) {
          if (ess_k[k] < target) {
            first = k + 1;
            break;
          }
        }
        const double nlo = lo + (hi - lo) * (first - 1) / K;
        const double nhi = first <= ninner ? lo + (hi - lo) * first / K : hi;
        ss.lo = nlo;
        ss.hi = nhi;
        if (r == rounds - 1) {
          ss.D = nlo > 0.0 ? nlo : nhi;
          ss.done = 1;
        }
      }
    }
    __syncthreads();
  }
  // the final reweighting at D (k_final_max, k_final_sum, k_normalise: nb blocks)
  const double a = ss.a, D = ss.D, h = 0.5 * ((a + D) * (a + D) - a * a);
  const int fstride = nb * blockDim.x;
  if (bid < nb) {
    double m0 = -INFINITY, m1 = -INFINITY;
    for (int i = bid * blockDim.x + tid; i < N; i += fstride) {
      const double lw = logW[i];
      m0 = fmax(m0, fma(-h, sig2[i], fma(D, ell[i], lw)));
      m1 = fmax(m1, lw);
    }
    w1[tid] = m0;
    w2[tid] = m1;
    tree_max2(w1, w2);
    if (tid == 0) {
      pmax[2 * bid] = w1[0];
      pmax[2 * bid + 1] = w2[0];
    }
  }
  if (!grid_barrier(st, nblk, &flag)) return;
  double M0, M1;
  {
    double m0 = -INFINITY, m1 = -INFINITY;
    for (int b = tid; b < nb; b += blockDim.x) {
      m0 = fmax(m0, __ldcg(pmax + 2 * b));
      m1 = fmax(m1, __ldcg(pmax + 2 * b + 1));
    }
    w1[tid] = m0;
    w2[tid] = m1;
    tree_max2(w1, w2);
    M0 = w1[0];
    M1 = w2[0];
    __syncthreads();
  }
  if (bid < nb) {
    double s1 = 0.0, s2 = 0.0, so = 0.0;
    for (int i = bid * blockDim.x + tid; i < N; i += fstride) {
      const double lw = logW[i];
      const double e = exp(fma(-h, sig2[i], fma(D, ell[i], lw)) - M0);
      s1 += e;
      s2 = fma(e, e, s2);
      so += exp(lw - M1);
    }
    w1[tid] = s1;
    w2[tid] = s2;
    w3[tid] = so;
    tree_sum3(w1, w2, w3);
    if (tid == 0) {
      psum[3 * bid] = w1[0];
      psum[3 * bid + 1] = w2[0];
      psum[3 * bid + 2] = w3[0];
    }
  }
  if (!grid_barrier(st, nblk, &flag)) return;
  {
    double s1 = 0.0, s2 = 0.0, so = 0.0;
    for (int b = tid; b < nb; b += blockDim.x) {
      s1 += __ldcg(psum + 3 * b);
      s2 += __ldcg(psum + 3 * b + 1);
      so += __ldcg(psum + 3 * b + 2);
    }
    w1[tid] = s1;
    w2[tid] = s2;
    w3[tid] = so;
    tree_sum3(w1, w2, w3);
  }
  const double t1 = w1[0], t2 = w2[0], to = w3[0];
  const double lse_new = M0 + log(t1), lse_old = M1 + log(to);
  if (bid == 0 && tid == 0) {  // the device state, as the separate launches leave it
    st->dmax = ss.dmax;
    st->lo = ss.lo;
    st->hi = ss.hi;
    st->best_dist = ss.best_dist;
    st->best_D = ss.best_D;
    st->D = D;
    st->search_done = 1;
    st->lse_new = lse_new;
    st->lse_old = lse_old;
    st->ess = t1 * t1 / t2;
    st->log_z_inc = lse_new - lse_old;
    st->log_z += st->log_z_inc;
    st->a_prev = a;
    st->a = (D == ss.dmax) ? 1.0 : a + D;
    if (!isfinite(lse_new) || !isfinite(lse_old)) atomicOr(&st->err, kErrNonFinite);
  }
  // normalised weights (every block; the reads of log W above are finished everywhere)
  for (int i = bid * blockDim.x + tid; i < N; i += nblk * blockDim.x) {
    const double l = fma(-h, sig2[i], fma(D, ell[i], logW[i])) - lse_new;
    logW[i] = l;
    W[i] = exp(l);
  }
}

int reweight(int N, const double *ell, const double *sig2, double *logW, double *W, double tau,
             int K, int rounds, int grid_points, double grid_decades, DevState *st,
             double *partials, int *launches, cudaStream_t s, bool one_launch) {
  if (grid_points > 0) {  // the grid in rounds of kMaxK points
    if (grid_points < 2 || !(grid_decades > 0.0)) return (int)cudaErrorInvalidValue;
    K = kMaxK;
    rounds = (grid_points + kMaxK - 1) / kMaxK;
  }
  if (K < 2 || K > kMaxK) return (int)cudaErrorInvalidValue;
  int nb = (N + kFinThreads - 1) / kFinThreads;
  if (nb > kRwMaxBlocks) nb = kRwMaxBlocks;
  int nbs = (N + 15) / 16;  // search: at least two particles per stream of 16 lanes
  if (nbs > kRwMaxBlocks) nbs = kRwMaxBlocks;
  double *gmax = partials;                     // [kMaxK]
  double *pmax = gmax + kMaxK;                 // [nbs][kMaxK]
  double *psum = pmax + kRwMaxBlocks * kMaxK;  // [nbs][kMaxK][2]
  if (one_launch) {  // every block resident at once: at most 152 blocks of 128 threads
    const int grid = nbs > nb ? nbs : nb;
    k_reweight_one<<<grid, kSwThreads, 0, s>>>(N, ell, sig2, logW, W, tau, K, rounds,
                                               grid_points, grid_decades, st, partials, nbs, nb);
    if (launches) *launches += 1;
    return (int)cudaGetLastError();
  }
  int count = 0;
  k_search_begin<<<1, 1, 0, s>>>(st);
  ++count;
  for (int r = 0; r < rounds; ++r) {
    k_search_max<<<nbs, kSwThreads, 0, s>>>(N, ell, sig2, logW, K, r, grid_points, grid_decades,
                                            st, pmax, gmax);
    k_search_sum<<<nbs, kSwThreads, 0, s>>>(N, ell, sig2, logW, tau, K, r, rounds - 1,
                                            grid_points, grid_decades, st, gmax, psum);
    count += 2;
  }
  k_final_max<<<nb, kFinThreads, 0, s>>>(N, ell, sig2, logW, st, pmax, gmax);
  k_final_sum<<<nb, kFinThreads, 0, s>>>(N, ell, sig2, logW, st, gmax, psum);
  k_normalise<<<nb, kFinThreads, 0, s>>>(N, ell, sig2, logW, W, st);
  count += 3;
  if (launches) *launches += count;
  return (int)cudaGetLastError();
}

// Doubles of scratch the temperature search needs.
int reweight_scratch_doubles() { return kMaxK + kRwMaxBlocks * kMaxK * 3; }

// ------------------------------------------------------------------------------------------------
// Weighted particle moments (Algorithm 2 (d)): mean = sum W_i theta_i, then
// Sigma = sum W_i (theta_i - mean)(theta_i - mean)'. FP64, block partials summed in block order.
// ------------------------------------------------------------------------------------------------
constexpr int kMomThreads = 256, kMomBlocks = 152;

template <typename CT>
__device__ __forceinline__ void k_mean_partials_body(int N, int p, const double *W, const CT *theta,
    double *part, int bid_, int nblk_) {
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    double s = 0.0;
    for (int i = bid_; i < N; i += nblk_) s += W[i] * (double)theta[(int64_t)i * p + c];
    part[(int64_t)bid_ * p + c] = s;
  }
}
template <typename CT>
__global__ void k_mean_partials(int N, int p, const double *W, const CT *theta, double *part) {
  k_mean_partials_body<CT>(N, p, W, theta, part, blockIdx.x, gridDim.x);
}
__device__ __forceinline__ void k_sum_partials_body(const double *part, int nblk, int width,
    double *out, int symmetric_p, int bid_, int nblk_) {
  const int lane = threadIdx.x & 31;
  const int warps = (nblk_ * blockDim.x) >> 5;
  for (int e = (bid_ * blockDim.x + threadIdx.x) >> 5; e < width; e += warps) {
    if (symmetric_p && e % symmetric_p < e / symmetric_p) continue;  // lower triangle: mirrored
    double s = 0.0;
    for (int b = lane; b < nblk; b += 32) s += part[(int64_t)b * width + e];
    s = warp_sum(s);
    if (lane != 0) continue;
    if (symmetric_p) {
      const int r = e / symmetric_p, c = e % symmetric_p;
      out[r * symmetric_p + c] = s;
      out[c * symmetric_p + r] = s;
    } else {
      out[e] = s;
    }
  }
}
__global__ void k_sum_partials(const double *part, int nblk, int width, double *out,
                               int symmetric_p) {
  k_sum_partials_body(part, nblk, width, out, symmetric_p, blockIdx.x, gridDim.x);
}
template <typename CT>
__device__ __forceinline__ void k_cov_partials_body(int N, int p, const double *W, const CT *theta,
    const double *mean, double *part, int bid_, int nblk_) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int r = e / p, c = e % p;
    if (c < r) continue;
    double s = 0.0;
    for (int i = bid_; i < N; i += nblk_) {
      const double dr = (double)theta[(int64_t)i * p + r] - mean[r];
      const double dc = (double)theta[(int64_t)i * p + c] - mean[c];
      s += W[i] * dr * dc;
    }
    part[(int64_t)bid_ * p * p + e] = s;
  }
}
template <typename CT>
__global__ void k_cov_partials(int N, int p, const double *W, const CT *theta, const double *mean,
                               double *part) {
  k_cov_partials_body<CT>(N, p, W, theta, mean, part, blockIdx.x, gridDim.x);
}

int weighted_moments(int is_f64, int N, int p, const double *W, const void *theta,
                     double *partials, double *mean, double *Sigma, cudaStream_t s) {
  const int nb = N < kMomBlocks ? N : kMomBlocks;
  if (is_f64)
    k_mean_partials<double><<<nb, 128, 0, s>>>(N, p, W, (const double *)theta, partials);
  else
    k_mean_partials<float><<<nb, 128, 0, s>>>(N, p, W, (const float *)theta, partials);
  k_sum_partials<<<(p + 7) / 8, 256, 0, s>>>(partials, nb, p, mean, 0);
  if (is_f64)
    k_cov_partials<double><<<nb, kMomThreads, 0, s>>>(N, p, W, (const double *)theta, mean,
                                                      partials);
  else
    k_cov_partials<float><<<nb, kMomThreads, 0, s>>>(N, p, W, (const float *)theta, mean,
                                                     partials);
  k_sum_partials<<<(p * p + 7) / 8, 256, 0, s>>>(partials, nb, p * p, Sigma, p);
  return (int)cudaGetLastError();
}

// Mass matrix: Cholesky of Sigma with the jitter schedule 1e-10 tr/p, x10 per retry (added
// cumulatively, at most 12 retries); then Linv = chol^{-1} for drawing rho = Linv' z. When no
// retry succeeds (e.g. a single particle: Sigma = 0) the previous mass matrix is kept.
template <typename CT>
__device__ __forceinline__ void k_mass_body(int p, const double *Sigma_in, double *Sigma,
    double *chol, CT *Sigma_ct, CT *Linv_ct, double *work, DevState *st, int bid_, int nblk_) {
  extern __shared__ double M[];
  __shared__ int flag;
  __shared__ double jit;
  const int tid = threadIdx.x;
  for (int e = tid; e < p * p; e += blockDim.x) work[e] = Sigma_in[e];
  if (tid == 0) {
    double tr = 0.0;
    for (int c = 0; c < p; ++c) tr += Sigma_in[c * p + c];
    jit = 1e-10 * tr / p;
  }
  __syncthreads();
  int tries = 0;
  bool ok = false;
  while (true) {
    for (int e = tid; e < p * p; e += blockDim.x) M[e] = work[e];
    __syncthreads();
    ok = chol_block(M, p, &flag);
    if (ok || tries == 12) break;
    ++tries;
    __syncthreads();
    for (int c = tid; c < p; c += blockDim.x) work[c * p + c] += jit;
    __syncthreads();
    if (tid == 0) jit *= 10.0;
    __syncthreads();
  }
  if (tid == 0) st->chol_retries = ok ? tries : -1;
  if (!ok) return;  // keep the previous mass matrix
  for (int e = tid; e < p * p; e += blockDim.x) {
    Sigma[e] = work[e];
    chol[e] = M[e];
    Sigma_ct[e] = (CT)work[e];
  }
  __syncthreads();
  // column j of Linv by forward substitution, L X = I (FP64 in work; each thread owns columns)
  for (int j = tid; j < p; j += blockDim.x) {
    for (int i = 0; i < j; ++i) work[i * p + j] = 0.0;
    work[j * p + j] = 1.0 / M[j * p + j];
    for (int i = j + 1; i < p; ++i) {
      double acc = 0.0;
      for (int k = j; k < i; ++k) acc += M[i * p + k] * work[k * p + j];
      work[i * p + j] = -acc / M[i * p + i];
    }
  }
  __syncthreads();
  for (int e = tid; e < p * p; e += blockDim.x) Linv_ct[e] = (CT)work[e];
}
template <typename CT>
__global__ void k_mass(int p, const double *Sigma_in, double *Sigma, double *chol, CT *Sigma_ct,
                       CT *Linv_ct, double *work, DevState *st) {
  k_mass_body<CT>(p, Sigma_in, Sigma, chol, Sigma_ct, Linv_ct, work, st, blockIdx.x, gridDim.x);
}

int mass_matrix(int is_f64, int p, const double *Sigma_in, double *Sigma, double *chol,
                void *Sigma_ct, void *Linv_ct, double *work, DevState *st, cudaStream_t s) {
  const size_t smem = (size_t)p * p * sizeof(double);
  cudaError_t e;
  if (is_f64) {
    e = cudaFuncSetAttribute(k_mass<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return (int)e;
    k_mass<double><<<1, 256, smem, s>>>(p, Sigma_in, Sigma, chol, (double *)Sigma_ct,
                                        (double *)Linv_ct, work, st);
  } else {
    e = cudaFuncSetAttribute(k_mass<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return (int)e;
    k_mass<float><<<1, 256, smem, s>>>(p, Sigma_in, Sigma, chol, (float *)Sigma_ct,
                                       (float *)Linv_ct, work, st);
  }
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Resampling (Algorithm 2 (e)) on integer weights w_i = floor(W_i 2^40): inclusive prefix sums
// cum (exact), T = cum[N-1]. Systematic: offset floor(U T) with U from the stage's resampling
// stream, position i = floor((i T + offset) / N). Multinomial (the paper's scheme, Sec. 2.2):
// position i = min(floor(U_i T), T - 1) with U_i from offspring i's own draw. Either way the
// ancestor is the first j with cum[j] > position.
// ------------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__device__ __forceinline__ void k_res_scan_body(int N, const double *W, uint64_t *cum,
    uint64_t seed, int stage, int stage_dev, DevState *st, int bid_, int nblk_) {
  __shared__ unsigned long long tot[kScanThreads];
  const int tid = threadIdx.x;
  const int per = (N + kScanThreads - 1) / kScanThreads;
  const int i0 = tid * per, i1 = min(N, i0 + per);
  unsigned long long s = 0;
  for (int i = i0; i < i1; ++i) s += (unsigned long long)floor(W[i] * 0x1.0p40);
  tot[tid] = s;
  __syncthreads();
  for (int o = 1; o < kScanThreads; o <<= 1) {  // Hillis-Steele inclusive scan of block totals
    const unsigned long long v = tid >= o ? tot[tid - o] : 0ull;
    __syncthreads();
    tot[tid] += v;
    __syncthreads();
  }
  unsigned long long run = tid ? tot[tid - 1] : 0ull;
  for (int i = i0; i < i1; ++i) {
    run += (unsigned long long)floor(W[i] * 0x1.0p40);
    cum[i] = run;
  }
  if (tid == kScanThreads - 1) {
    const unsigned long long T = tot[kScanThreads - 1];
    const Stream rs(seed, kResample, stage_move(stage_dev ? st->stage : stage, 0), 0u);
    const double U = draw_uniform(rs.draw(0));
    st->res_T = T;
    st->res_off = (unsigned long long)floor(U * (double)T);
  }
}
__global__ void __launch_bounds__(kScanThreads)
    k_res_scan(int N, const double *W, uint64_t *cum, uint64_t seed, int stage, int stage_dev,
               DevState *st) {
  k_res_scan_body(N, W, cum, seed, stage, stage_dev, st, blockIdx.x, gridDim.x);
}

__device__ __forceinline__ void k_res_ancestors_body(int N, const uint64_t *cum, int32_t *anc,
    const DevState *st, uint64_t seed, int stage, int stage_dev, int multinomial, int bid_,
    int nblk_) {
  const unsigned long long T = st->res_T, off = st->res_off;
  const uint32_t sm = stage_move(stage_dev ? st->stage : stage, 0);
  for (int i = bid_ * blockDim.x + threadIdx.x; i < N; i += nblk_ * blockDim.x) {
    if (T == 0) {
      anc[i] = i;
      continue;
    }
    unsigned long long pos;
    if (multinomial) {
      const double Ui = draw_uniform(Stream(seed, kResample, sm, (uint32_t)i).draw(1));
      pos = (unsigned long long)floor(Ui * (double)T);
      if (pos > T - 1) pos = T - 1;
    } else {
      pos = ((unsigned long long)i * T + off) / (unsigned long long)N;
    }
    int lo = 0, hi = N - 1;  // first j with cum[j] > pos; cum[N-1] = T > pos
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (cum[mid] > pos)
        hi = mid;
      else
        lo = mid + 1;
    }
    anc[i] = lo;
  }
}
__global__ void k_res_ancestors(int N, const uint64_t *cum, int32_t *anc, const DevState *st,
                                uint64_t seed, int stage, int stage_dev, int multinomial) {
  k_res_ancestors_body(N, cum, anc, st, seed, stage, stage_dev, multinomial, blockIdx.x, gridDim.x);
}

template <typename CT>
__device__ __forceinline__ void k_res_gather_body(int N, int p, int m, int G, const int32_t *anc,
    const CT *theta, CT *theta_out, const int32_t *u, int32_t *u_out, const double *ell,
    double *ell_out, const double *sig2, double *sig2_out, const double *blk, double *blk_out,
    double *logW, double *W, int bid_, int nblk_) {
  const int warp = (bid_ * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (nblk_ * blockDim.x) >> 5;
  for (int i = warp; i < N; i += nwarps) {
    const int a = anc[i];
    for (int c = lane; c < p; c += 32) theta_out[(int64_t)i * p + c] = theta[(int64_t)a * p + c];
    const int32_t *us = u + (int64_t)a * m;
    int32_t *ud = u_out + (int64_t)i * m;
    if ((m & 3) == 0) {
      const int4 *s4 = reinterpret_cast<const int4 *>(us);
      int4 *d4 = reinterpret_cast<int4 *>(ud);
      for (int j = lane; j < m / 4; j += 32) d4[j] = s4[j];
    } else {
      for (int j = lane; j < m; j += 32) ud[j] = us[j];
    }
    for (int h = lane; h < 2 * G; h += 32)
      blk_out[(int64_t)i * 2 * G + h] = blk[(int64_t)a * 2 * G + h];
    if (lane == 0) {
      ell_out[i] = ell[a];
      sig2_out[i] = sig2[a];
      logW[i] = -log((double)N);
      W[i] = 1.0 / (double)N;
    }
  }
}
template <typename CT>
__global__ void k_res_gather(int N, int p, int m, int G, const int32_t *anc, const CT *theta,
                             CT *theta_out, const int32_t *u, int32_t *u_out, const double *ell,
                             double *ell_out, const double *sig2, double *sig2_out,
                             const double *blk, double *blk_out, double *logW, double *W) {
  k_res_gather_body<CT>(N, p, m, G, anc, theta, theta_out, u, u_out, ell, ell_out, sig2, sig2_out,
                        blk, blk_out, logW, W, blockIdx.x, gridDim.x);
}

int resample(int is_f64, int N, int p, int m, int G, uint64_t seed, int stage, int stage_dev,
             int multinomial, const double *W, uint64_t *cum, int32_t *anc, const void *theta, void *theta_out, const int32_t *u,
             int32_t *u_out, const double *ell, double *ell_out, const double *sig2,
             double *sig2_out, const double *blk, double *blk_out, double *logW, double *Wout,
             DevState *st, cudaStream_t s) {
  k_res_scan<<<1, kScanThreads, 0, s>>>(N, W, cum, seed, stage, stage_dev, st);
  k_res_ancestors<<<(N + 255) / 256, 256, 0, s>>>(N, cum, anc, st, seed, stage, stage_dev,
                                                   multinomial);
  const int gw = (N * 32 + 255) / 256;
  const int grid = gw < 152 * 16 ? gw : 152 * 16;
  if (is_f64)
    k_res_gather<double><<<grid, 256, 0, s>>>(N, p, m, G, anc, (const double *)theta,
                                              (double *)theta_out, u, u_out, ell, ell_out, sig2,
                                              sig2_out, blk, blk_out, logW, Wout);
  else
    k_res_gather<float><<<grid, 256, 0, s>>>(N, p, m, G, anc, (const float *)theta,
                                             (float *)theta_out, u, u_out, ell, ell_out, sig2,
                                             sig2_out, blk, blk_out, logW, Wout);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Small helpers
// ------------------------------------------------------------------------------------------------
__global__ void k_weights_from(int N, const double *Win, double *logW, double *W) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double w = Win ? Win[i] : 1.0 / (double)N;
    W[i] = w;
    logW[i] = Win ? log(w) : -log((double)N);
  }
}
int weights_from(int N, const double *W_in, double *logW, double *W, cudaStream_t s) {
  k_weights_from<<<(N + 255) / 256, 256, 0, s>>>(N, W_in, logW, W);
  return (int)cudaGetLastError();
}

__device__ __forceinline__ void k_eps_update_body(int N, int R, double target, DevState *st,
    int bid_, int nblk_) {
  const double rate = (double)st->acc_theta / ((double)N * (double)R);
  const double f = exp(rate - target);
  st->eps *= f < 0.5 ? 0.5 : (f > 2.0 ? 2.0 : f);
}
__global__ void k_eps_update(int N, int R, double target, DevState *st) {
  k_eps_update_body(N, R, target, st, blockIdx.x, gridDim.x);
}
int eps_update(int N, int R, DevState *st, cudaStream_t s, double target) {
  k_eps_update<<<1, 1, 0, s>>>(N, R, target, st);
  return (int)cudaGetLastError();
}

// Componentwise correlation across particles between two clouds (the stage's starting cloud and
// the current one), for the adaptive number of moves: one block per component, FP64, two passes
// (means, then centred sums), fixed reduction order. A component with no spread in either cloud
// gets correlation 1.
constexpr int kAcThreads = 256;
__device__ __forceinline__ double block_sum_fixed(double v, double *sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
  for (int w = 0; w < kAcThreads / 32; ++w) t += sh[w];
  return t;
}
template <typename CT>
__global__ void __launch_bounds__(kAcThreads)
    k_autocorr(int N, int p, const CT *a, const CT *b, double *rho) {
  __shared__ double sh[kAcThreads / 32];
  const int c = blockIdx.x;
  double sa = 0.0, sb = 0.0;
  for (int i = threadIdx.x; i < N; i += kAcThreads) {
    sa += (double)a[(int64_t)i * p + c];
    sb += (double)b[(int64_t)i * p + c];
  }
  const double ma = block_sum_fixed(sa, sh) / N;
  const double mb = block_sum_fixed(sb, sh) / N;
  double xx = 0.0, yy = 0.0, xy = 0.0;
  for (int i = threadIdx.x; i < N; i += kAcThreads) {
    const double dx = (double)a[(int64_t)i * p + c] - ma, dy = (double)b[(int64_t)i * p + c] - mb;
    xx = fma(dx, dx, xx);
    yy = fma(dy, dy, yy);
    xy = fma(dx, dy, xy);
  }
  xx = block_sum_fixed(xx, sh);
  yy = block_sum_fixed(yy, sh);
  xy = block_sum_fixed(xy, sh);
  if (threadIdx.x == 0) rho[c] = (xx > 0.0 && yy > 0.0) ? xy / sqrt(xx * yy) : 1.0;
}
int autocorr(int is_f64, int N, int p, const void *a, const void *b, double *rho, cudaStream_t s) {
  if (is_f64)
    k_autocorr<double><<<p, kAcThreads, 0, s>>>(N, p, (const double *)a, (const double *)b, rho);
  else
    k_autocorr<float><<<p, kAcThreads, 0, s>>>(N, p, (const float *)a, (const float *)b, rho);
  return (int)cudaGetLastError();
}

template <typename CT> __global__ void k_convert(int count, const double *src, CT *dst) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    dst[i] = (CT)src[i];
}
int to_state_type(int is_f64, int count, const double *src, void *dst, cudaStream_t s) {
  const int grid = (count + 255) / 256 < 1024 ? (count + 255) / 256 : 1024;
  if (count <= 0) return 0;
  if (is_f64)
    k_convert<double><<<grid, 256, 0, s>>>(count, src, (double *)dst);
  else
    k_convert<float><<<grid, 256, 0, s>>>(count, src, (float *)dst);
  return (int)cudaGetLastError();
}
__global__ void k_round_f32(int count, double *v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    v[i] = (double)(float)v[i];
}
int round_to_state_type(int is_f64, int count, double *v, cudaStream_t s) {
  if (is_f64 || count <= 0) return 0;
  k_round_f32<<<(count + 255) / 256, 256, 0, s>>>(count, v);
  return (int)cudaGetLastError();
}

}  // namespace subsmc

namespace subsmc {
namespace {
__global__ void k_stage_set(DevState *st, int stage) { st->stage = stage; }
__global__ void k_stage_advance(DevState *st) { st->stage += 1; }
}  // namespace

int stage_set(DevState *st, int stage, cudaStream_t s) {
  k_stage_set<<<1, 1, 0, s>>>(st, stage);
  return (int)cudaGetLastError();
}

int stage_advance(DevState *st, cudaStream_t s) {
  k_stage_advance<<<1, 1, 0, s>>>(st);
  return (int)cudaGetLastError();
}

}  // namespace subsmc

// ------------------------------------------------------------------------------------------------
// The stage steps of a batch of problems in a few launches: every kernel body above runs for
// problem q on blocks off[kind][q] .. off[kind][q + 1] - 1 of one launch, with q's own block count
// (that of its single-problem launch), so each problem's reductions run in the same order as when
// it is stepped alone.
// ------------------------------------------------------------------------------------------------
namespace subsmc {

int stage_kind_blocks(int kind, int N, int p) {
  switch (kind) {
    case kSkSearch: return N + 15 < 16 * kRwMaxBlocks ? (N + 15) / 16 : kRwMaxBlocks;
    case kSkFinal: {
      const int nb = (N + kFinThreads - 1) / kFinThreads;
      return nb < kRwMaxBlocks ? nb : kRwMaxBlocks;
    }
    case kSkMom: return N < kMomBlocks ? N : kMomBlocks;
    case kSkSumMean: return (p + 7) / 8;
    case kSkSumCov: return (p * p + 7) / 8;
    case kSkAnc: return (N + 255) / 256;
    case kSkGather: {
      const int gw = (N * 32 + 255) / 256;
      return gw < 152 * 16 ? gw : 152 * 16;
    }
    default: return 0;
  }
}

namespace {

__device__ __forceinline__ int stage_kind_blocks_dev(int kind, int N) {
  return kind == kSkMom ? (N < kMomBlocks ? N : kMomBlocks) : 0;
}

// the problem that owns block g: the last q with off[q] <= g
__device__ __forceinline__ int problem_of(const int *off, int P, int g) {
  int lo = 0, hi = P - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

struct Slot {
  const StageArgs *a;
  int bid, nblk;
};
__device__ __forceinline__ Slot slot_of(const StageArgs *A, const int *off, int P) {
  const int q = problem_of(off, P, (int)blockIdx.x);
  return Slot{A + q, (int)blockIdx.x - off[q], off[q + 1] - off[q]};
}

// partial scratch of a problem: [kMaxK] maxima | [kRwMaxBlocks][kMaxK] | [kRwMaxBlocks][kMaxK][2]
__device__ __forceinline__ double *gmax_of(const StageArgs &a) { return a.part; }
__device__ __forceinline__ double *pmax_of(const StageArgs &a) { return a.part + kMaxK; }
__device__ __forceinline__ double *psum_of(const StageArgs &a) {
  return a.part + kMaxK + kRwMaxBlocks * kMaxK;
}

// one thread per problem: stage counter, accept counters, search bracket
__global__ void kb_begin(const StageArgs *A, int P) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  DevState *st = A[q].st;
  st->stage += 1;
  st->acc_u = 0ull;
  st->acc_theta = 0ull;
  k_search_begin_body(st, 0, 1);
}

__global__ void __launch_bounds__(kSwThreads)
    kb_search_max(const StageArgs *A, const int *off, int P, int round) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_search_max_body(a.N, a.ell, a.sig2, a.logW, a.K, round, a.S, a.E, a.st, pmax_of(a), gmax_of(a),
                    s.bid, s.nblk);
}
__global__ void __launch_bounds__(kSwThreads)
    kb_search_sum(const StageArgs *A, const int *off, int P, int round) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_search_sum_body(a.N, a.ell, a.sig2, a.logW, a.tau, a.K, round, a.last_round, a.S, a.E, a.st,
                    gmax_of(a), psum_of(a), s.bid, s.nblk);
}
__global__ void __launch_bounds__(kFinThreads)
    kb_final_max(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_final_max_body(a.N, a.ell, a.sig2, a.logW, a.st, pmax_of(a), gmax_of(a), s.bid, s.nblk);
}
__global__ void __launch_bounds__(kFinThreads)
    kb_final_sum(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_final_sum_body(a.N, a.ell, a.sig2, a.logW, a.st, gmax_of(a), psum_of(a), s.bid, s.nblk);
}
__global__ void kb_normalise(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_normalise_body(a.N, a.ell, a.sig2, a.logW, a.W, a.st, s.bid, s.nblk);
}
__global__ void kb_mean_partials(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_mean_partials_body<float>(a.N, a.p, a.W, a.theta, a.part, s.bid, s.nblk);
}
__global__ void kb_sum_mean(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_sum_partials_body(a.part, stage_kind_blocks_dev(kSkMom, a.N), a.p, a.mean, 0, s.bid, s.nblk);
}
__global__ void kb_cov_partials(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_cov_partials_body<float>(a.N, a.p, a.W, a.theta, a.mean, a.part, s.bid, s.nblk);
}
__global__ void kb_sum_cov(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_sum_partials_body(a.part, stage_kind_blocks_dev(kSkMom, a.N), a.p * a.p, a.Sigma_raw, a.p,
                      s.bid, s.nblk);
}
__global__ void kb_mass(const StageArgs *A) {
  const StageArgs &a = A[blockIdx.x];
  k_mass_body<float>(a.p, a.Sigma_raw, a.Sigma, a.chol, a.Sigma_ct, a.Linv_ct, a.work, a.st, 0, 1);
}
__global__ void __launch_bounds__(kScanThreads) kb_res_scan(const StageArgs *A) {
  const StageArgs &a = A[blockIdx.x];
  k_res_scan_body(a.N, a.W, a.cum, a.seed, 0, 1, a.st, 0, 1);
}
__global__ void kb_res_ancestors(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_res_ancestors_body(a.N, a.cum, a.anc, a.st, a.seed, 0, 1, a.multinomial, s.bid, s.nblk);
}
__global__ void kb_res_gather(const StageArgs *A, const int *off, int P) {
  const Slot s = slot_of(A, off, P);
  const StageArgs &a = *s.a;
  k_res_gather_body<float>(a.N, a.p, a.m, a.G, a.anc, a.theta, a.theta_out, a.u, a.u_out, a.ell,
                           a.ell_out, a.sig2, a.sig2_out, a.blk, a.blk_out, a.logW, a.W, s.bid,
                           s.nblk);
}
__global__ void kb_eps_update(const StageArgs *A, int P, int R) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P) return;
  const StageArgs &a = A[q];
  k_eps_update_body(a.N, R, a.eps_target, a.st, 0, 1);
}

}  // namespace

int stage_batch(const StageBatch &sb, cudaStream_t s, int64_t *launches) {
  const int P = sb.P;
  auto off = [&](int kind) { return sb.off + (size_t)kind * (P + 1); };
  int64_t nl = 0;
  kb_begin<<<(P + 127) / 128, 128, 0, s>>>(sb.args, P);
  ++nl;
  for (int r = 0; r < sb.max_rounds; ++r) {
    kb_search_max<<<sb.total[kSkSearch], kSwThreads, 0, s>>>(sb.args, off(kSkSearch), P, r);
    kb_search_sum<<<sb.total[kSkSearch], kSwThreads, 0, s>>>(sb.args, off(kSkSearch), P, r);
    nl += 2;
  }
  kb_final_max<<<sb.total[kSkFinal], kFinThreads, 0, s>>>(sb.args, off(kSkFinal), P);
  kb_final_sum<<<sb.total[kSkFinal], kFinThreads, 0, s>>>(sb.args, off(kSkFinal), P);
  kb_normalise<<<sb.total[kSkFinal], kFinThreads, 0, s>>>(sb.args, off(kSkFinal), P);
  kb_mean_partials<<<sb.total[kSkMom], 128, 0, s>>>(sb.args, off(kSkMom), P);
  kb_sum_mean<<<sb.total[kSkSumMean], 256, 0, s>>>(sb.args, off(kSkSumMean), P);
  kb_cov_partials<<<sb.total[kSkMom], kMomThreads, 0, s>>>(sb.args, off(kSkMom), P);
  kb_sum_cov<<<sb.total[kSkSumCov], 256, 0, s>>>(sb.args, off(kSkSumCov), P);
  const size_t smem = (size_t)sb.max_p * sb.max_p * sizeof(double);
  cudaError_t e =
      cudaFuncSetAttribute(kb_mass, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return (int)e;
  kb_mass<<<P, 256, smem, s>>>(sb.args);
  kb_res_scan<<<P, kScanThreads, 0, s>>>(sb.args);
  kb_res_ancestors<<<sb.total[kSkAnc], 256, 0, s>>>(sb.args, off(kSkAnc), P);
  kb_res_gather<<<sb.total[kSkGather], 256, 0, s>>>(sb.args, off(kSkGather), P);
  nl += 11;
  if (launches) *launches += nl;
  return (int)cudaGetLastError();
}

int eps_update_batch(const StageBatch &sb, int R, cudaStream_t s) {
  kb_eps_update<<<(sb.P + 127) / 128, 128, 0, s>>>(sb.args, sb.P, R);
  return (int)cudaGetLastError();
}

}  // namespace subsmc
