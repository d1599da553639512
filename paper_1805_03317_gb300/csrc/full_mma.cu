// Full-data log-likelihood and gradient for many particles on the tensor cores: the comparison
// method of the paper's experiments (Sec. 4: full-data SMC), with
//   l(theta_i) = sum_k l_k(x_k'theta_i),   grad l(theta_i) = sum_k l'_k(x_k'theta_i) x_k
// for every particle i and all n rows. Both sums are dense contractions: per CTA, a tile of 128
// particles walks tiles of 128 rows and runs, per row tile,
//   GEMM1  E[i, k] = sum_c Theta[i, c] X[k, c]          (M = 128 particles, N = 128 rows, K = p)
//   epilogue: one thread per particle reads its 128 etas from tensor memory, forms l_k and l'_k
//           (FP32, fast exponential/logarithm), accumulates l in FP64 and writes l'_k as two BF16
//           terms (hi + lo) into shared memory
//   GEMM2  G[i, c] += sum_k P[i, k] X[k, c]              (M = 128, N = p padded, K = 128 rows)
// with tcgen05.mma (kind::f16, FP32 accumulators in tensor memory). X is exact in BF16; theta is
// split into three BF16 terms so eta keeps FP32 accuracy. The X tile in shared memory serves
// both GEMMs: it is the K-major B operand of GEMM1 and the MN-major B operand of GEMM2 (same bytes,
// different descriptors). CTAs split the rows into chunks; per-particle sums are combined with
// FP64 atomics, and a finishing kernel adds the per-row constants, the prior and the temperature.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace subsmc {
namespace {

constexpr int kP = 128;          // particles per CTA = MMA M = threads
constexpr int kR = 128;          // rows per tile = GEMM1 N = GEMM2 K
constexpr int kStrip = 16 * 128; // bytes of one 8-column (or 8-row) strip over 128 rows/particles
constexpr long long kWaitCycles = 4000000000ll;
// Extra shared memory past the operand tiles (none: the descriptors' layouts are checked by the
// parity tests; a nonzero guard keeps a mistaken stride inside the CTA's allocation).
constexpr int kGuard = 0;

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// No-swizzle shared-memory matrix descriptor: LBO = byte stride between core matrices adjacent in
// K, SBO = between core matrices adjacent in M/N; bits 46-48 = 0b001.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// kind::f16, FP32 accumulator, BF16 operands; a_mn / b_mn: operand is MN-major.
__host__ __device__ constexpr uint32_t idesc(int M, int N, int a_mn, int b_mn) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(id), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          su32(bar))
      : "memory");
}
__device__ __forceinline__ bool try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on an mbarrier phase; false (on every thread) if any thread ran out of time.
__device__ __forceinline__ bool wait_phase(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  bool done = try_wait(bar, parity);
  while (!done && clock64() - t0 < kWaitCycles) done = try_wait(bar, parity);
  return __syncthreads_and(done) != 0;
}
__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void fence_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void ld16(uint32_t taddr, float *v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int e = 0; e < 16; ++e) v[e] = __uint_as_float(r[e]);
}
__device__ __forceinline__ uint32_t bf(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bfv(uint32_t b) { return __uint_as_float(b << 16); }

// Offset of unit (index t in 0..127, 8-wide chunk q) in a 128 x (8 * chunks) tile: chunk strips
// of kStrip bytes, 8-index core matrices of 128 bytes, 16 bytes per index.
__device__ __forceinline__ int uoff(int t, int q) { return q * kStrip + (t >> 3) * 128 + (t & 7) * 16; }

// theta-dependent part of l_k and its eta-derivative, FP32 (the per-row constants of the Poisson,
// Gaussian and Student-t log-densities are added once per particle by the finishing kernel).
template <int FAM>
__device__ __forceinline__ void fam_terms(float eta, float y, float inv_s2, float nu, float &l,
                                          float &d1) {
  if (FAM == 4) {  // Student-t: -(nu+1)/2 log(1 + r^2 / (nu s^2)), (nu+1) r / (nu s^2 + r^2)
    const float r = y - eta, z = r * r * inv_s2;
    l = -0.5f * (nu + 1.f) * log1pf(z / nu);
    d1 = __fdividef((nu + 1.f) * r * inv_s2, nu + z);
  } else if (FAM == 0) {  // logistic: y eta - softplus(eta), y - sigma(eta)
    const float e = __expf(-fabsf(eta));
    const float inv = __fdividef(1.f, 1.f + e);
    l = y * eta - (fmaxf(eta, 0.f) + __logf(1.f + e));
    d1 = y - (eta >= 0.f ? inv : e * inv);
  } else if (FAM == 2) {  // Poisson: y eta - e^eta
    const float mu = __expf(eta);
    l = y * eta - mu;
    d1 = y - mu;
  } else if (FAM == 3) {  // Gaussian: -(y - eta)^2 / (2 sigma^2)
    const float r = y - eta;
    l = -0.5f * r * r * inv_s2;
    d1 = r * inv_s2;
  } else {  // probit: log Phi(s eta), s lambda(s eta)
    const float s = 2.f * y - 1.f;
    float lp, lam;
    log_phi_(s * eta, lp, lam);
    l = lp;
    d1 = s * lam;
  }
}

__device__ __forceinline__ void cp4(void *smem, const void *gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(su32(smem)), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(su32(smem)), "l"(gmem)
               : "memory");
}

// l'_k of 8 consecutive rows as BF16 hi and lo terms, packed for the K-major P tile.
__device__ __forceinline__ void split8(const float *d, uint4 &hi, uint4 &lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const __nv_bfloat162 hb = __floats2bfloat162_rn(d[2 * q], d[2 * q + 1]);
    const float2 hf = __bfloat1622float2(hb);
    const __nv_bfloat162 lb = __floats2bfloat162_rn(d[2 * q] - hf.x, d[2 * q + 1] - hf.y);
    h[q] = *reinterpret_cast<const uint32_t *>(&hb);
    l[q] = *reinterpret_cast<const uint32_t *>(&lb);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// 256 threads: warps w and w + 4 share the TMEM lane quadrant w (particles 32w .. 32w + 31) and
// split a row tile's 128 columns into halves. Row tiles are double-buffered: the next tile's
// copies are in flight during the current epilogue, and GEMM1 of a tile overlaps GEMM2 of the
// previous one on the tensor pipe.
constexpr int kThreads = 256;

template <int FAM>
__global__ void __launch_bounds__(kThreads) k_full_mma(
    const __nv_bfloat16 *Xp, int64_t n, int p, int S, int Yo, float inv_s2, float nu,
    const float *theta,
    int B, int ntile_p, int nchunk, int64_t chunk_rows, double *acc, int Kp, int Np, int *flag) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  const int kq = Kp / 8;  // 8-column chunks of a row (GEMM1 K)
  unsigned char *Xt = sm;                        // 2 buffers x [kq strips][128 rows]
  unsigned char *Th = Xt + 2 * kq * kStrip;      // 3 terms x [kq strips][128 particles]
  unsigned char *Pt = Th + 3 * kq * kStrip;      // 2 terms x [16 strips][128 particles]
  float *ys = reinterpret_cast<float *>(Pt + 2 * 16 * kStrip);  // 2 x [128] responses
  uint64_t *bar = reinterpret_cast<uint64_t *>(ys + 2 * kR);
  uint32_t *tptr = reinterpret_cast<uint32_t *>(bar + 2);

  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;\n" ::"r"(
                     su32(tptr))
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tptr, tE = tmem, tG = tmem + 128;
  const uint32_t tlane = (uint32_t)(quad * 32) << 16;
  const uint32_t id1 = idesc(kP, kR, 0, 0), id2 = idesc(kP, Np, 0, 1);
  const uint32_t xb = su32(Xt), thb = su32(Th), pb = su32(Pt);
  uint32_t ph1 = 0, ph2 = 0;
  bool ok = true;
  const int items = ntile_p * nchunk;
  // copies of the row tile starting at row t0 into buffer b (rows past r1 are zero)
  auto load_tile = [&](int64_t t0, int64_t r1, int b) {
    unsigned char *xt = Xt + b * kq * kStrip;
    for (int u = tid; u < kR * kq; u += kThreads) {
      const int k = u / kq, q = u - k * kq;
      unsigned char *dst = xt + uoff(k, q);
      if (t0 + k < r1 && 8 * q < p)
        cp16(dst, Xp + (t0 + k) * S + 8 * q);
      else
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    if (tid < kR) {
      if (t0 + tid < r1)
        cp4(ys + b * kR + tid, &reinterpret_cast<const RowC<float> *>(Xp + (t0 + tid) * S + Yo)->y);
      else
        ys[b * kR + tid] = 0.f;
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };
  for (int item = blockIdx.x; item < items && ok; item += gridDim.x) {
    const int pt = item / nchunk, ch = item - pt * nchunk;
    const int i0 = pt * kP;
    const int64_t r0 = ch * chunk_rows, r1 = min(n, r0 + chunk_rows);
    // theta of the particle tile as three BF16 terms, K-major (unit = 8 columns of a particle)
    if (tid < kP) {
      const int i = i0 + tid;
      for (int q = 0; q < kq; ++q) {
        uint32_t h[8], m_[8], l_[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int c = 8 * q + e;
          const float v = (i < B && c < p) ? theta[(int64_t)i * p + c] : 0.f;
          h[e] = bf(v);
          const float r1_ = v - bfv(h[e]);
          m_[e] = bf(r1_);
          l_[e] = bf(r1_ - bfv(m_[e]));
        }
        const int off = uoff(tid, q);
        *reinterpret_cast<uint4 *>(Th + off) =
            make_uint4(h[0] | h[1] << 16, h[2] | h[3] << 16, h[4] | h[5] << 16, h[6] | h[7] << 16);
        *reinterpret_cast<uint4 *>(Th + kq * kStrip + off) = make_uint4(
            m_[0] | m_[1] << 16, m_[2] | m_[3] << 16, m_[4] | m_[5] << 16, m_[6] | m_[7] << 16);
        *reinterpret_cast<uint4 *>(Th + 2 * kq * kStrip + off) = make_uint4(
            l_[0] | l_[1] << 16, l_[2] | l_[3] << 16, l_[4] | l_[5] << 16, l_[6] | l_[7] << 16);
      }
    }
    load_tile(r0, r1, 0);
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    fence_async();
    fence_before();
    __syncthreads();
    const int i = i0 + quad * 32 + lane;  // this thread's particle
    const bool live = i < B;
    const bool full_p = i0 + kP <= B;
    double lsum = 0.0;
    int j = 0;
    for (int64_t t0 = r0; t0 < r1; t0 += kR, ++j) {
      const int b = j & 1;
      // 1. GEMM1 of this tile: E = Theta X'
      if (tid == 0) {
        fence_after();
        for (int s = 0; s < 3; ++s)
          for (int kk = 0; kk < Kp / 16; ++kk) {
            const uint64_t ad = desc(thb + s * kq * kStrip + kk * 2 * kStrip, kStrip, 128);
            const uint64_t bd = desc(xb + b * kq * kStrip + kk * 2 * kStrip, kStrip, 128);
            mma(tE, ad, bd, id1, (s > 0 || kk > 0) ? 1u : 0u);
          }
        commit(bar);
      }
      // 2. GEMM2 of the previous tile must be done before its X buffer and P are reused
      if (j > 0) {
        ok = wait_phase(bar + 1, ph2);
        ph2 ^= 1u;
        fence_after();
      }
      // 3. copies of the next tile, in flight during the epilogue
      if (ok && t0 + kR < r1) load_tile(t0 + kR, r1, b ^ 1);
      const bool okE = wait_phase(bar, ph1);
      ph1 ^= 1u;
      fence_after();
      if (!ok || !okE) {
        ok = false;
        break;
      }
      // 4. epilogue: l and l' of this thread's particle over its half of the tile's rows
      {
        const float *yt = ys + b * kR;
        const bool fast = full_p && t0 + kR <= r1;
        for (int c0 = half * 64; c0 < half * 64 + 64; c0 += 16) {
          float v[16], d[16];
          ld16(tE + tlane + (uint32_t)c0, v);
          const float4 y4[4] = {*reinterpret_cast<const float4 *>(yt + c0),
                                *reinterpret_cast<const float4 *>(yt + c0 + 4),
                                *reinterpret_cast<const float4 *>(yt + c0 + 8),
                                *reinterpret_cast<const float4 *>(yt + c0 + 12)};
          const float *yy = reinterpret_cast<const float *>(y4);
          float ls = 0.f;
#pragma unroll
          for (int e = 0; e < 16; ++e) {
            float l = 0.f;
            d[e] = 0.f;
            if (fast || (live && t0 + c0 + e < r1)) fam_terms<FAM>(v[e], yy[e], inv_s2, nu, l, d[e]);
            ls += l;
          }
          lsum += (double)ls;
          uint4 hi0, lo0, hi1, lo1;
          split8(d, hi0, lo0);
          split8(d + 8, hi1, lo1);
          const int q0 = c0 / 8, pr = quad * 32 + lane;
          *reinterpret_cast<uint4 *>(Pt + uoff(pr, q0)) = hi0;
          *reinterpret_cast<uint4 *>(Pt + uoff(pr, q0 + 1)) = hi1;
          *reinterpret_cast<uint4 *>(Pt + 16 * kStrip + uoff(pr, q0)) = lo0;
          *reinterpret_cast<uint4 *>(Pt + 16 * kStrip + uoff(pr, q0 + 1)) = lo1;
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");  // the next tile has landed
      fence_async();
      fence_before();
      __syncthreads();
      // 5. GEMM2: G += P X (P terms hi, lo), K = 128 rows; X as the MN-major B operand
      if (tid == 0) {
        fence_after();
        for (int s = 0; s < 2; ++s)
          for (int kk = 0; kk < kR / 16; ++kk) {
            const uint64_t ad = desc(pb + s * 16 * kStrip + kk * 2 * kStrip, kStrip, 128);
            const uint64_t bd = desc(xb + b * kq * kStrip + kk * 256, 128, kStrip);
            mma(tG, ad, bd, id2, (j > 0 || s > 0 || kk > 0) ? 1u : 0u);
          }
        commit(bar + 1);
      }
    }
    if (ok && j > 0) {  // the last GEMM2
      ok = wait_phase(bar + 1, ph2);
      ph2 ^= 1u;
      fence_after();
    }
    // 6. the item's sums into its own slot acc[chunk][i][0..p] (summed over chunks in a fixed
    // order by the finishing kernel, so results do not depend on scheduling): l from both
    // halves (half 1 first, through shared memory), G from half 0
    double *slot = acc + ((int64_t)ch * B + i) * (p + 1);
    double *lred = reinterpret_cast<double *>(Th);  // theta tiles are free until the next item
    __syncthreads();
    if (half == 1) lred[quad * 32 + lane] = lsum;
    __syncthreads();
    if (ok && j > 0 && half == 0) {
      if (live) slot[0] = lsum + lred[quad * 32 + lane];
      for (int c0 = 0; c0 < Np; c0 += 16) {
        float v[16];
        ld16(tG + tlane + (uint32_t)c0, v);
        if (live) {
#pragma unroll
          for (int e = 0; e < 16; ++e)
            if (c0 + e < p) slot[1 + c0 + e] = (double)v[e];
        }
      }
    }
    fence_before();
    __syncthreads();  // theta tiles and the accumulators are reused by the next item
  }
  if (!ok && tid == 0) atomicExch(flag, 1);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;\n" ::"r"(tmem)
                 : "memory");
  }
}

// ell[i] = l + constant; grad[i] = a * grad l - (theta - mu) / v (state type); a from *a_dev
// when given (the device temperature), else a_host.
__global__ void k_full_finish(int B, int p, int nchunk, const double *acc, double lconst,
                              double a_host, const double *a_dev, const float *theta,
                              const float *mu, const float *ivar, double *ell, float *grad) {
  const double a = a_dev ? *a_dev : a_host;
  const int64_t per = (int64_t)B * (p + 1);
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per;
       e += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int q = 0; q < nchunk; ++q) t += acc[q * per + e];  // chunk order: deterministic
    const int64_t i = e / (p + 1);
    const int c = (int)(e - i * (p + 1));
    if (c == 0) {
      if (ell) ell[i] = t + lconst;
    } else if (grad) {
      const int j = c - 1;
      grad[i * p + j] = (float)(a * t) - (theta[i * p + j] - mu[j]) * ivar[j];
    }
  }
}

// Sum over rows of the theta-free part of the log-density: -lgamma(y + 1) (Poisson),
// -log(2 pi sigma^2) / 2 (Gaussian) or lgamma((nu+1)/2) - lgamma(nu/2) - log(nu pi s^2) / 2
// (Student-t); FP64, per-block partial sums added atomically.
__global__ void k_full_const(const __nv_bfloat16 *Xp, int64_t n, int S, int Yo, int fam, double s2,
                             double nu, double *out) {
  const double tc = fam == 4 ? lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) -
                                   0.5 * log(3.14159265358979323846 * nu * s2)
                             : 0.0;
  double t = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n;
       k += (int64_t)gridDim.x * blockDim.x) {
    const double y = (double)reinterpret_cast<const RowC<float> *>(Xp + k * S + Yo)->y;
    if (fam == 2) t -= lgamma(y + 1.0);
    if (fam == 3) t -= 0.5 * log(6.283185307179586476925286766559 * s2);
    if (fam == 4) t += tc;
  }
  t = warp_sum(t);
  if ((threadIdx.x & 31) == 0 && t != 0.0) atomicAdd(out, t);
}

size_t full_smem(int Kp) {
  return (size_t)(Kp / 8) * kStrip * 5 + (size_t)2 * 16 * kStrip + 2 * kR * sizeof(float) + 32 +
         kGuard;
}

// Row chunks per particle tile for B particles over n rows (the number of accumulator slots).
int full_chunks(int64_t n, int B, int sms, int64_t *chunk_rows_out) {
  const int ntile = (B + kP - 1) / kP;
  const int slots = 2 * sms;
  int nchunk = (slots + ntile - 1) / ntile;
  const int64_t max_chunks = (n + kR - 1) / kR;
  if (nchunk > max_chunks) nchunk = (int)max_chunks;
  if (nchunk < 1) nchunk = 1;
  int64_t chunk_rows = (n + nchunk - 1) / nchunk;
  chunk_rows = ((chunk_rows + kR - 1) / kR) * kR;
  if (chunk_rows_out) *chunk_rows_out = chunk_rows;
  return (int)((n + chunk_rows - 1) / chunk_rows);
}

template <int FAM>
int launch_full(const __nv_bfloat16 *Xp, int64_t n, int p, int S, int Yo, float inv_s2, float nu,
                const float *theta, int B, double *acc, int *flag, int sms, cudaStream_t s) {
  const int Kp = ((p + 15) / 16) * 16, Np = ((p + 15) / 16) * 16;
  const size_t smem = full_smem(Kp);
  cudaError_t e = cudaFuncSetAttribute(k_full_mma<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  cudaFuncSetAttribute(k_full_mma<FAM>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_full_mma<FAM>, kThreads, smem);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  // Two CTAs per SM (256 tensor-memory columns each). CTAs never wait for one another, so a grid
  // larger than what is resident simply runs in waves.
  per_sm = 2;
  const int slots = per_sm * sms;
  const int ntile = (B + kP - 1) / kP;
  int64_t chunk_rows = 0;
  const int nchunk = full_chunks(n, B, sms, &chunk_rows);
  const int items = ntile * nchunk;
  const int grid = items < slots ? items : slots;
  k_full_mma<FAM><<<grid, kThreads, smem, s>>>(Xp, n, p, S, Yo, inv_s2, nu, theta, B, ntile,
                                               nchunk, chunk_rows, acc, Kp, Np, flag);
  return (int)cudaGetLastError();
}

}  // namespace

int full_acc_doubles(int64_t n, int p, int B, int sms) {
  return full_chunks(n, B, sms, nullptr) * B * (p + 1);
}

int full_loglik_const(const void *Xp, int64_t n, int S, int Yo, int fam, double sigma2, double nu,
                      double *out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double), s);
  if (e != cudaSuccess) return (int)e;
  if (fam != 2 && fam != 3 && fam != 4) return 0;
  k_full_const<<<152 * 4, 256, 0, s>>>((const __nv_bfloat16 *)Xp, n, S, Yo, fam, sigma2, nu, out);
  return (int)cudaGetLastError();
}

int full_loglik(const void *Xp, int64_t n, int p, int S, int Yo, int fam, double sigma2, double nu,
                const void *theta, int B, double a, const double *a_dev, double lconst,
                const void *mu, const void *ivar, double *acc, int *flag, double *ell, void *grad,
                int sms, cudaStream_t s) {
  if (p < 1 || p > 64 || B < 0) return (int)cudaErrorInvalidValue;
  if (B == 0) return 0;
  // every (chunk, live particle) slot of acc is written by exactly one CTA item
  const __nv_bfloat16 *X = (const __nv_bfloat16 *)Xp;
  const float *th = (const float *)theta;
  const float i2 = (float)(1.0 / sigma2), v = (float)nu;
  int r;
  switch (fam) {
    case 0: r = launch_full<0>(X, n, p, S, Yo, i2, v, th, B, acc, flag, sms, s); break;
    case 1: r = launch_full<1>(X, n, p, S, Yo, i2, v, th, B, acc, flag, sms, s); break;
    case 2: r = launch_full<2>(X, n, p, S, Yo, i2, v, th, B, acc, flag, sms, s); break;
    case 3: r = launch_full<3>(X, n, p, S, Yo, i2, v, th, B, acc, flag, sms, s); break;
    default: r = launch_full<4>(X, n, p, S, Yo, i2, v, th, B, acc, flag, sms, s); break;
  }
  if (r) return r;
  const int64_t tot = (int64_t)B * (p + 1);
  const int grid = (int)((tot + 255) / 256 < 152 * 8 ? (tot + 255) / 256 : 152 * 8);
  k_full_finish<<<grid, 256, 0, s>>>(B, p, full_chunks(n, B, sms, nullptr), acc, lconst, a, a_dev,
                                     th, (const float *)mu, (const float *)ivar, ell,
                                     (float *)grad);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// HMC move of the full-data comparison SMC (Algorithm 1 step 2 with the exact log-likelihood): one
// warp per particle, columns lane and lane + 32 (p <= 64). The leapfrog loop between fm_begin and
// fm_accept is kicks and drifts around full_loglik evaluations; the random numbers (momentum,
// MH uniform) use the same Philox streams as the subsampled trajectory kernels.
// ------------------------------------------------------------------------------------------------
namespace {

struct Cols {  // a particle's p values held two per lane
  float v0, v1;
};
__device__ __forceinline__ float col_get(const Cols &x, int c) {
  const float a = __shfl_sync(0xffffffffu, x.v0, c & 31), b = __shfl_sync(0xffffffffu, x.v1, c & 31);
  return c < 32 ? a : b;
}
// (M x)_r for r = lane, lane + 32 with M [p, p] row-major symmetric-use: sum_k M[k * p + r] x_k
__device__ __forceinline__ Cols matvec(const float *M, const Cols &x, int p, int lane) {
  Cols o{0.f, 0.f};
  for (int k = 0; k < p; ++k) {
    const float xk = col_get(x, k);
    if (lane < p) o.v0 = fmaf(M[k * p + lane], xk, o.v0);
    if (lane + 32 < p) o.v1 = fmaf(M[k * p + lane + 32], xk, o.v1);
  }
  return o;
}
__device__ __forceinline__ double half_quad(const Cols &x, const Cols &Mx, int p, int lane) {
  double t = 0.0;
  if (lane < p) t += (double)x.v0 * (double)Mx.v0;
  if (lane + 32 < p) t += (double)x.v1 * (double)Mx.v1;
  return 0.5 * warp_sum(t);
}
__device__ __forceinline__ double log_prior_cols(const float *th, const float *mu, const float *iv,
                                                 int p, int lane) {
  double t = 0.0;
  for (int c = lane; c < p; c += 32) {
    const double r = (double)th[c] - (double)mu[c];
    t += -0.5 * r * r * (double)iv[c];
  }
  return warp_sum(t);
}

__global__ void k_fm_begin(int N, int p, const float *theta, float *thp, float *rho,
                           const float *Linv, const float *Sigma, const float *mu,
                           const float *ivar, const double *ell, uint64_t seed, int stage,
                           int stage_dev, int move, const DevState *st, double *h0,
                           double jitter, float *eps_out) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  const uint32_t sm = stage_move(stage_dev ? st->stage : stage, move);
  if (lane == 0) eps_out[i] = (float)jittered_eps(st->eps, jitter, seed, sm, (uint32_t)i);
  const Stream smom(seed, kMomentum, sm, (uint32_t)i);
  Cols z{0.f, 0.f};
  if (lane < p) z.v0 = (float)stream_normal(smom, (uint32_t)lane);
  if (lane + 32 < p) z.v1 = (float)stream_normal(smom, (uint32_t)(lane + 32));
  Cols r{0.f, 0.f};  // rho_r = sum_{c >= r} Linv[c, r] z_c
  for (int c = 0; c < p; ++c) {
    const float zc = col_get(z, c);
    if (lane < p && c >= lane) r.v0 = fmaf(Linv[c * p + lane], zc, r.v0);
    if (lane + 32 < p && c >= lane + 32) r.v1 = fmaf(Linv[c * p + lane + 32], zc, r.v1);
  }
  const float *th = theta + (int64_t)i * p;
  for (int c = lane; c < p; c += 32) thp[(int64_t)i * p + c] = th[c];
  if (lane < p) rho[(int64_t)i * p + lane] = r.v0;
  if (lane + 32 < p) rho[(int64_t)i * p + lane + 32] = r.v1;
  const double kin = half_quad(r, matvec(Sigma, r, p, lane), p, lane);
  const double lp = log_prior_cols(th, mu, ivar, p, lane);
  if (lane == 0) h0[i] = -(st->a * ell[i] + lp) + kin;
}

// rho += eps_i/2 g; then, if drift, theta += eps_i Sigma rho (eps_i: the particle's step size,
// written by k_fm_begin).
__global__ void k_fm_kick(int N, int p, float *thp, float *rho, const float *g, const float *Sigma,
                          const float *eps_i, int drift) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  const float eps = eps_i[i];
  float *r = rho + (int64_t)i * p;
  const float *gi = g + (int64_t)i * p;
  Cols x{0.f, 0.f};
  if (lane < p) x.v0 = r[lane] + 0.5f * eps * gi[lane];
  if (lane + 32 < p) x.v1 = r[lane + 32] + 0.5f * eps * gi[lane + 32];
  if (lane < p) r[lane] = x.v0;
  if (lane + 32 < p) r[lane + 32] = x.v1;
  if (drift) {
    const Cols v = matvec(Sigma, x, p, lane);
    float *t = thp + (int64_t)i * p;
    if (lane < p) t[lane] += eps * v.v0;
    if (lane + 32 < p) t[lane + 32] += eps * v.v1;
  }
}

__global__ void k_fm_accept(int N, int p, float *theta, const float *thp, const float *rho,
                            const float *Sigma, const float *mu, const float *ivar, double *ell,
                            const double *ell_new, const double *h0, uint64_t seed, int stage,
                            int stage_dev, int move, DevState *st) {
  const int lane = threadIdx.x & 31;
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (i >= N) return;
  Cols r{0.f, 0.f};
  if (lane < p) r.v0 = rho[(int64_t)i * p + lane];
  if (lane + 32 < p) r.v1 = rho[(int64_t)i * p + lane + 32];
  const double kin = half_quad(r, matvec(Sigma, r, p, lane), p, lane);
  const float *t = thp + (int64_t)i * p;
  const double lp = log_prior_cols(t, mu, ivar, p, lane);
  const double h1 = -(st->a * ell_new[i] + lp) + kin;
  const Stream smh(seed, kMhTheta, stage_move(stage_dev ? st->stage : stage, move), (uint32_t)i);
  const double U = draw_uniform(smh.draw(0));
  const bool acc = log(U) < h0[i] - h1;  // false when h1 is NaN
  if (acc) {
    for (int c = lane; c < p; c += 32) theta[(int64_t)i * p + c] = t[c];
    if (lane == 0) {
      ell[i] = ell_new[i];
      atomicAdd(&st->acc_theta, 1ull);
    }
  }
}

}  // namespace

int full_move_begin(int N, int p, const void *theta, void *thp, void *rho, const void *Linv,
                    const void *Sigma, const void *mu, const void *ivar, const double *ell,
                    uint64_t seed, int stage, int stage_dev, int move, const DevState *st,
                    double *h0, double jitter, float *eps_out, cudaStream_t s) {
  k_fm_begin<<<(N * 32 + 255) / 256, 256, 0, s>>>(
      N, p, (const float *)theta, (float *)thp, (float *)rho, (const float *)Linv,
      (const float *)Sigma, (const float *)mu, (const float *)ivar, ell, seed, stage, stage_dev,
      move, st, h0, jitter, eps_out);
  return (int)cudaGetLastError();
}

int full_move_kick(int N, int p, void *thp, void *rho, const void *g, const void *Sigma,
                   const float *eps_i, int drift, cudaStream_t s) {
  k_fm_kick<<<(N * 32 + 255) / 256, 256, 0, s>>>(N, p, (float *)thp, (float *)rho,
                                                   (const float *)g, (const float *)Sigma, eps_i,
                                                   drift);
  return (int)cudaGetLastError();
}

int full_move_accept(int N, int p, void *theta, const void *thp, const void *rho,
                     const void *Sigma, const void *mu, const void *ivar, double *ell,
                     const double *ell_new, const double *h0, uint64_t seed, int stage,
                     int stage_dev, int move, DevState *st, cudaStream_t s) {
  k_fm_accept<<<(N * 32 + 255) / 256, 256, 0, s>>>(
      N, p, (float *)theta, (const float *)thp, (const float *)rho, (const float *)Sigma,
      (const float *)mu, (const float *)ivar, ell, ell_new, h0, seed, stage, stage_dev, move, st);
  return (int)cudaGetLastError();
}

}  // namespace subsmc
