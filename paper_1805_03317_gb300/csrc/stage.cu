// Stage-level kernels of subsampling SMC (Algorithm 2): data packing, control-variate moments
// (Sec. 3.2), the Newton step for the control-variate centre, particle initialisation, the
// temperature search and reweighting (Sec. 2.2, Sec. 3.3, Sec. 3.5), weighted moments and the mass
// matrix (Algorithm 2 (d)), and systematic resampling (Algorithm 2 (e)).
#include <cuda_bf16.h>
#include <math.h>

#include "device.cuh"
#include "internal.h"

namespace subsmc {

namespace {

__device__ __forceinline__ double warp_sum_d(double v) { return warp_sum(v); }

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

// (max, s1, s2) triples of an online log-sum-exp of x and 2x: s1 = sum e^{x-max}, s2 = sum e^{2(x-max)}.
struct Lse {
  double m, s1, s2;
  __device__ __forceinline__ Lse() : m(-INFINITY), s1(0.0), s2(0.0) {}
  __device__ __forceinline__ void add(double x) {
    if (!(x > -INFINITY)) return;  // zero weight (or NaN: flagged by the caller)
    if (x > m) {
      const double r = exp(m - x);
      s1 = s1 * r + 1.0;
      s2 = s2 * r * r + 1.0;
      m = x;
    } else {
      const double e = exp(x - m);
      s1 += e;
      s2 += e * e;
    }
  }
  __device__ __forceinline__ void merge(const Lse &o) {
    if (!(o.m > -INFINITY)) return;
    if (!(m > -INFINITY)) {
      *this = o;
      return;
    }
    if (o.m > m) {
      const double r = exp(m - o.m);
      s1 = s1 * r + o.s1;
      s2 = s2 * r * r + o.s2;
      m = o.m;
    } else {
      const double r = exp(o.m - m);
      s1 += o.s1 * r;
      s2 += o.s2 * r * r;
    }
  }
  __device__ __forceinline__ Lse shfl_xor(int o) const {
    Lse t;
    t.m = __shfl_xor_sync(0xffffffffu, m, o);
    t.s1 = __shfl_xor_sync(0xffffffffu, s1, o);
    t.s2 = __shfl_xor_sync(0xffffffffu, s2, o);
    return t;
  }
};

__device__ Lse block_lse(Lse v, Lse *red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
  for (int o = 16; o; o >>= 1) v.merge(v.shfl_xor(o));
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  Lse t;
  for (int k = 0; k < nw; ++k) t.merge(red[k]);
  return t;
}

template <typename CT> __device__ __forceinline__ double ld_state(const void *p, int64_t i) {
  return (double)reinterpret_cast<const CT *>(p)[i];
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Packing: row k of Xp = [y_k | x_k | 0 ...], stride S elements. y is stored in the first 8 (FP64)
// or 4 (otherwise) bytes of the row.
// ------------------------------------------------------------------------------------------------
template <typename E, typename YT>
__global__ void k_pack(const E *X, int64_t n, int p, int64_t ld, const YT *y, E *Xp, int S) {
  constexpr int YS = sizeof(YT) / sizeof(E);
  const int64_t total = n * (int64_t)S;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = t / S;
    const int s = (int)(t - k * S);
    E v;
    if (s < YS) {
      const YT yk = y[k];
      v = reinterpret_cast<const E *>(&yk)[s];
    } else if (s - YS < p) {
      v = X[k * ld + (s - YS)];
    } else {
      v = E(0);
    }
    Xp[t] = v;
  }
}

int pack_rows(const void *X, int x_dtype, int64_t n, int p, int64_t ld, const void *y, void *Xp,
              int S, cudaStream_t s) {
  const int64_t total = n * (int64_t)S;
  const int grid = (int)((total + 255) / 256 < 152 * 32 ? (total + 255) / 256 : 152 * 32);
  if (x_dtype == 0)
    k_pack<uint64_t, double><<<grid, 256, 0, s>>>((const uint64_t *)X, n, p, ld,
                                                  (const double *)y, (uint64_t *)Xp, S);
  else if (x_dtype == 1)
    k_pack<uint32_t, float><<<grid, 256, 0, s>>>((const uint32_t *)X, n, p, ld, (const float *)y,
                                                (uint32_t *)Xp, S);
  else
    k_pack<uint16_t, float><<<grid, 256, 0, s>>>((const uint16_t *)X, n, p, ld, (const float *)y,
                                                (uint16_t *)Xp, S);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Control-variate moments at theta (Sec. 3.2), FP64: A = sum_k l_k, B = sum_k l'_k x_k,
// C = sum_k l''_k x_k x_k'. Each block takes tiles of 32 rows; its threads own fixed (r, c) pairs
// of the upper triangle. Block partials are summed in block order by a second kernel.
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
template <typename XT> __device__ __forceinline__ double packed_y(const XT *row) {
  if (sizeof(XT) == 8) return *reinterpret_cast<const double *>(row);
  return (double)*reinterpret_cast<const float *>(row);
}

template <typename XT>
__global__ void __launch_bounds__(kCvThreads) k_cv_partials(const XT *Xp, int64_t n, int p, int S,
                                                            int fam, double s2,
                                                            const double *theta, double *part) {
  constexpr int YS = sizeof(XT) == 8 ? 1 : 4 / (int)sizeof(XT);
  extern __shared__ double sh[];
  double *xs = sh;                    // [kCvTile][p]
  double *wx = xs + kCvTile * p;      // [kCvTile][p]   l'' * x
  double *d1s = wx + kCvTile * p;     // [kCvTile]
  double *ths = d1s + kCvTile;        // [p]
  double *red = ths + p;              // [32]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int np = p * (p + 1) / 2;
  for (int c = tid; c < p; c += blockDim.x) ths[c] = theta[c];
  int qr[kCvMaxPairs], qc[kCvMaxPairs];
  double acc[kCvMaxPairs];
#pragma unroll
  for (int i = 0; i < kCvMaxPairs; ++i) {
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
    for (int rr = warp; rr < kCvTile; rr += kCvThreads / 32) {
      const int64_t k = k0 + rr;
      double eta = 0.0;
      if (k < n) {
        const XT *row = Xp + k * S;
        for (int c = lane; c < p; c += 32) {
          const double x = packed_x<XT>(row, YS + c);
          xs[rr * p + c] = x;
          eta += x * ths[c];
        }
      } else {
        for (int c = lane; c < p; c += 32) xs[rr * p + c] = 0.0;
      }
      eta = warp_sum_d(eta);
      double l = 0.0, d1 = 0.0, d2 = 0.0;
      if (k < n) {
        const double y = packed_y<XT>(Xp + k * S);
        switch (fam) {
          case 0: row_value<0>(eta, y, s2, l, d1, d2); break;
          case 1: row_value<1>(eta, y, s2, l, d1, d2); break;
          case 2: row_value<2>(eta, y, s2, l, d1, d2); break;
          default: row_value<3>(eta, y, s2, l, d1, d2); break;
        }
      }
      if (lane == 0) {
        d1s[rr] = d1;
        Aacc += l;
      }
      __syncwarp();
      for (int c = lane; c < p; c += 32) wx[rr * p + c] = d2 * xs[rr * p + c];
    }
    __syncthreads();
    for (int rr = 0; rr < kCvTile; ++rr) {
#pragma unroll
      for (int i = 0; i < kCvMaxPairs; ++i)
        if (tid + i * kCvThreads < np) acc[i] = fma(wx[rr * p + qr[i]], xs[rr * p + qc[i]], acc[i]);
      if (tid < p) Bacc = fma(d1s[rr], xs[rr * p + tid], Bacc);
    }
    __syncthreads();
  }
  double *out = part + (int64_t)blockIdx.x * (1 + p + np);
  const double A = block_sum(Aacc, red);
  if (tid == 0) out[0] = A;
  if (tid < p) out[1 + tid] = Bacc;
#pragma unroll
  for (int i = 0; i < kCvMaxPairs; ++i) {
    const int q = tid + i * kCvThreads;
    if (q < np) out[1 + p + q] = acc[i];
  }
}

__global__ void k_cv_reduce(const double *part, int nblk, int p, double *A, double *B, double *C) {
  const int np = p * (p + 1) / 2, width = 1 + p + np;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * width + e];
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

int cv_moments_blocks(int p) {
  (void)p;
  return 2 * 152;
}

int cv_moments(const void *Xp, int x_dtype, int64_t n, int p, int S, int fam, double sigma2,
               const double *theta, double *partials, int nblocks, double *A, double *B,
               double *C, cudaStream_t s) {
  if (p * (p + 1) / 2 > kCvThreads * kCvMaxPairs) return (int)cudaErrorInvalidValue;
  const size_t smem = (size_t)(2 * kCvTile * p + kCvTile + p + 32) * sizeof(double);
  cudaError_t e;
  if (x_dtype == 0) {
    e = cudaFuncSetAttribute(k_cv_partials<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    k_cv_partials<double><<<nblocks, kCvThreads, smem, s>>>((const double *)Xp, n, p, S, fam,
                                                            sigma2, theta, partials);
  } else if (x_dtype == 1) {
    e = cudaFuncSetAttribute(k_cv_partials<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    k_cv_partials<float><<<nblocks, kCvThreads, smem, s>>>((const float *)Xp, n, p, S, fam,
                                                           sigma2, theta, partials);
  } else {
    e = cudaFuncSetAttribute(k_cv_partials<__nv_bfloat16>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cv_partials<__nv_bfloat16><<<nblocks, kCvThreads, smem, s>>>(
        (const __nv_bfloat16 *)Xp, n, p, S, fam, sigma2, theta, partials);
  }
  if (e != cudaSuccess) return (int)e;
  const int width = 1 + p + p * (p + 1) / 2;
  k_cv_reduce<<<(width + 255) / 256, 256, 0, s>>>(partials, nblocks, p, A, B, C);
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
  for (int e = tid; e < p * p; e += blockDim.x) {
    const int i = e / p, k = e % p;
    M[e] = -C[e] + (i == k ? 1.0 / var[i] : 0.0);
  }
  for (int c = tid; c < p; c += blockDim.x) g[c] = B[c] - (theta[c] - mu[c]) / var[c];
  __syncthreads();
  const bool ok = chol_block(M, p, &flag);
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
// with s1 = sum e^{lw - max}, s2 = sum e^{2(lw - max)}. Round -1 tests D = 1 - a; each later round
// evaluates the K-1 interior points of the bracket and keeps the first sub-interval whose right end
// has ESS < tau N. Partials of every block are merged in block order by the last block to finish.
// ------------------------------------------------------------------------------------------------
constexpr int kRwThreads = 128, kMaxK = 32;

__device__ __forceinline__ double lw_at(double logW, double ell, double sig2, double a, double D) {
  return logW + D * ell - 0.5 * ((a + D) * (a + D) - a * a) * sig2;
}

__global__ void __launch_bounds__(kRwThreads)
    k_search_round(int N, const double *ell, const double *sig2, const double *logW, double tau,
                   int K, int round, int last_round, DevState *st, Lse *part) {
  __shared__ Lse red[kRwThreads / 32];
  __shared__ bool is_last;
  if (st->search_done) return;  // uniform across the grid
  const double a = st->a;
  const double lo = round < 0 ? 0.0 : st->lo, hi = round < 0 ? st->dmax : st->hi;
  const int ncand = round < 0 ? 1 : K - 1;
  for (int k = 0; k < ncand; ++k) {
    const double D = round < 0 ? hi : lo + (hi - lo) * (k + 1) / K;
    Lse acc;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x)
      acc.add(lw_at(logW[i], ell[i], sig2[i], a, D));
    acc = block_lse(acc, red);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * kMaxK + k] = acc;
  }
  __threadfence();
  if (threadIdx.x == 0) is_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __shared__ double ess_k[kMaxK];
  if (threadIdx.x < ncand) {  // one thread per candidate merges the block partials in order
    Lse t;
    for (int b = 0; b < (int)gridDim.x; ++b) t.merge(part[(int64_t)b * kMaxK + threadIdx.x]);
    ess_k[threadIdx.x] = t.s1 * t.s1 / t.s2;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const double target = tau * (double)N;
  int first = ncand + 1;  // 1-based index of the first candidate with ESS < target
  for (int k = 0; k < ncand; ++k) {
    const double ess = ess_k[k];
    if (!(ess == ess)) atomicOr(&st->err, kErrNonFinite);
    if (ess < target) {
      first = k + 1;
      break;
    }
  }
  if (round < 0) {
    if (first > ncand) {  // ESS(1 - a) >= target: go straight to a = 1
      st->D = st->dmax;
      st->search_done = 1;
    } else {
      st->lo = 0.0;
      st->hi = st->dmax;
    }
  } else {
    const double nlo = lo + (hi - lo) * (first - 1) / K;
    const double nhi = first <= ncand ? lo + (hi - lo) * first / K : hi;
    st->lo = nlo;
    st->hi = nhi;
    if (round == last_round) {
      st->D = nlo > 0.0 ? nlo : nhi;
      st->search_done = 1;
    }
  }
  st->ticket = 0;
}

// Final pass: log-sum-exps of the new and old log weights, ESS, log Z increment (Sec. 3.5).
__global__ void __launch_bounds__(kRwThreads)
    k_reweight_final(int N, const double *ell, const double *sig2, const double *logW,
                     DevState *st, Lse *part) {
  __shared__ Lse red[kRwThreads / 32];
  __shared__ bool is_last;
  const double a = st->a, D = st->D;
  Lse nw, ow;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    nw.add(lw_at(logW[i], ell[i], sig2[i], a, D));
    ow.add(logW[i]);
  }
  nw = block_lse(nw, red);
  ow = block_lse(ow, red);
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = nw;
    part[2 * blockIdx.x + 1] = ow;
  }
  __threadfence();
  if (threadIdx.x == 0) is_last = atomicAdd(&st->ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ Lse tot[2];
  if (threadIdx.x < 2) {
    Lse t;
    for (int b = 0; b < (int)gridDim.x; ++b) t.merge(part[2 * b + threadIdx.x]);
    tot[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  const Lse tn = tot[0], to = tot[1];
  const double lse_new = tn.m + log(tn.s1), lse_old = to.m + log(to.s1);
  st->lse_new = lse_new;
  st->lse_old = lse_old;
  st->ess = tn.s1 * tn.s1 / tn.s2;
  st->log_z_inc = lse_new - lse_old;
  st->log_z += st->log_z_inc;
  st->a_prev = a;
  st->a = (D == st->dmax) ? 1.0 : a + D;
  if (!isfinite(lse_new) || !isfinite(lse_old)) atomicOr(&st->err, kErrNonFinite);
  st->ticket = 0;
}

__global__ void k_normalise(int N, const double *ell, const double *sig2, double *logW, double *W,
                            const DevState *st) {
  const double a = st->a_prev, D = st->D, lse = st->lse_new;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const double l = lw_at(logW[i], ell[i], sig2[i], a, D) - lse;
    logW[i] = l;
    W[i] = exp(l);
  }
}

__global__ void k_search_begin(DevState *st) {
  st->dmax = 1.0 - st->a;
  st->lo = 0.0;
  st->hi = st->dmax;
  st->D = 0.0;
  st->search_done = 0;
  st->ticket = 0;
}

int reweight(int N, const double *ell, const double *sig2, double *logW, double *W, double tau,
             int K, int rounds, DevState *st, double *partials, int *launches, cudaStream_t s) {
  if (K < 2 || K > kMaxK) return (int)cudaErrorInvalidValue;
  int nb = (N + kRwThreads - 1) / kRwThreads;
  if (nb > 64) nb = 64;
  Lse *part = reinterpret_cast<Lse *>(partials);
  int count = 0;
  k_search_begin<<<1, 1, 0, s>>>(st);
  ++count;
  for (int r = -1; r < rounds; ++r) {
    k_search_round<<<nb, kRwThreads, 0, s>>>(N, ell, sig2, logW, tau, K, r, rounds - 1, st, part);
    ++count;
  }
  k_reweight_final<<<nb, kRwThreads, 0, s>>>(N, ell, sig2, logW, st, part);
  k_normalise<<<nb, kRwThreads, 0, s>>>(N, ell, sig2, logW, W, st);
  count += 2;
  if (launches) *launches += count;
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Weighted particle moments (Algorithm 2 (d)): mean = sum W_i theta_i, then
// Sigma = sum W_i (theta_i - mean)(theta_i - mean)'. FP64, block partials summed in block order.
// ------------------------------------------------------------------------------------------------
constexpr int kMomThreads = 256, kMomBlocks = 152;

template <typename CT>
__global__ void k_mean_partials(int N, int p, const double *W, const CT *theta, double *part) {
  for (int c = threadIdx.x; c < p; c += blockDim.x) {
    double s = 0.0;
    for (int i = blockIdx.x; i < N; i += gridDim.x) s += W[i] * (double)theta[(int64_t)i * p + c];
    part[(int64_t)blockIdx.x * p + c] = s;
  }
}
__global__ void k_sum_partials(const double *part, int nblk, int width, double *out,
                               int symmetric_p) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < width; e += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += part[(int64_t)b * width + e];
    if (symmetric_p) {
      const int r = e / symmetric_p, c = e % symmetric_p;
      if (c < r) continue;
      out[r * symmetric_p + c] = s;
      out[c * symmetric_p + r] = s;
    } else {
      out[e] = s;
    }
  }
}
template <typename CT>
__global__ void k_cov_partials(int N, int p, const double *W, const CT *theta, const double *mean,
                               double *part) {
  for (int e = threadIdx.x; e < p * p; e += blockDim.x) {
    const int r = e / p, c = e % p;
    if (c < r) continue;
    double s = 0.0;
    for (int i = blockIdx.x; i < N; i += gridDim.x) {
      const double dr = (double)theta[(int64_t)i * p + r] - mean[r];
      const double dc = (double)theta[(int64_t)i * p + c] - mean[c];
      s += W[i] * dr * dc;
    }
    part[(int64_t)blockIdx.x * p * p + e] = s;
  }
}

int weighted_moments(int is_f64, int N, int p, const double *W, const void *theta,
                     double *partials, double *mean, double *Sigma, cudaStream_t s) {
  const int nb = N < kMomBlocks ? N : kMomBlocks;
  if (is_f64)
    k_mean_partials<double><<<nb, 128, 0, s>>>(N, p, W, (const double *)theta, partials);
  else
    k_mean_partials<float><<<nb, 128, 0, s>>>(N, p, W, (const float *)theta, partials);
  k_sum_partials<<<1, 128, 0, s>>>(partials, nb, p, mean, 0);
  if (is_f64)
    k_cov_partials<double><<<nb, kMomThreads, 0, s>>>(N, p, W, (const double *)theta, mean,
                                                      partials);
  else
    k_cov_partials<float><<<nb, kMomThreads, 0, s>>>(N, p, W, (const float *)theta, mean,
                                                     partials);
  k_sum_partials<<<(p * p + 255) / 256, 256, 0, s>>>(partials, nb, p * p, Sigma, p);
  return (int)cudaGetLastError();
}

// Mass matrix: Cholesky of Sigma with the jitter schedule 1e-10 tr/p, x10 per retry (added
// cumulatively, at most 12 retries); then Linv = chol^{-1} for drawing rho = Linv' z. When no
// retry succeeds (e.g. a single particle: Sigma = 0) the previous mass matrix is kept.
template <typename CT>
__global__ void k_mass(int p, const double *Sigma_in, double *Sigma, double *chol, CT *Sigma_ct,
                       CT *Linv_ct, double *work, DevState *st) {
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
// Systematic resampling (Algorithm 2 (e)) on integer weights w_i = floor(W_i 2^40): inclusive
// prefix sums cum (exact), T = cum[N-1], offset floor(U T) with U from the stage's resampling
// stream, position i = floor((i T + offset) / N), ancestor = first j with cum[j] > position.
// ------------------------------------------------------------------------------------------------
constexpr int kScanThreads = 1024;

__global__ void __launch_bounds__(kScanThreads)
    k_res_scan(int N, const double *W, uint64_t *cum, uint64_t seed, int stage, DevState *st) {
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
    const Stream rs(seed, kResample, stage_move(stage, 0), 0u);
    const double U = draw_uniform(rs.draw(0));
    st->res_T = T;
    st->res_off = (unsigned long long)floor(U * (double)T);
  }
}

__global__ void k_res_ancestors(int N, const uint64_t *cum, int32_t *anc, const DevState *st) {
  const unsigned long long T = st->res_T, off = st->res_off;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    if (T == 0) {
      anc[i] = i;
      continue;
    }
    const unsigned long long pos = ((unsigned long long)i * T + off) / (unsigned long long)N;
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

template <typename CT>
__global__ void k_res_gather(int N, int p, int m, int G, const int32_t *anc, const CT *theta,
                             CT *theta_out, const int32_t *u, int32_t *u_out, const double *ell,
                             double *ell_out, const double *sig2, double *sig2_out,
                             const double *blk, double *blk_out, double *logW, double *W) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
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
    for (int h = lane; h < 2 * G; h += 32) blk_out[(int64_t)i * 2 * G + h] = blk[(int64_t)a * 2 * G + h];
    if (lane == 0) {
      ell_out[i] = ell[a];
      sig2_out[i] = sig2[a];
      logW[i] = -log((double)N);
      W[i] = 1.0 / (double)N;
    }
  }
}

int resample(int is_f64, int N, int p, int m, int G, uint64_t seed, int stage, const double *W,
             uint64_t *cum, int32_t *anc, const void *theta, void *theta_out, const int32_t *u,
             int32_t *u_out, const double *ell, double *ell_out, const double *sig2,
             double *sig2_out, const double *blk, double *blk_out, double *logW, double *Wout,
             DevState *st, cudaStream_t s) {
  k_res_scan<<<1, kScanThreads, 0, s>>>(N, W, cum, seed, stage, st);
  k_res_ancestors<<<(N + 255) / 256, 256, 0, s>>>(N, cum, anc, st);
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

__global__ void k_eps_update(int N, int R, DevState *st) {
  const double rate = (double)st->acc_theta / ((double)N * (double)R);
  const double f = exp(rate - 0.65);
  st->eps *= f < 0.5 ? 0.5 : (f > 2.0 ? 2.0 : f);
}
int eps_update(int N, int R, DevState *st, cudaStream_t s) {
  k_eps_update<<<1, 1, 0, s>>>(N, R, st);
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
