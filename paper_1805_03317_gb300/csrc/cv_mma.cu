// Control-variate moments on the tensor cores for BF16 storage (Sec. 3.2: A = sum_k l_k,
// B = sum_k l'_k x_k, C = sum_k l''_k x_k x_k', all at theta).
//
// C = X' diag(l'') X is a dense contraction over the n rows, so it runs as tcgen05 MMAs with the
// accumulator in tensor memory: per tile of 128 rows, D[i, j] += sum_k x_ki * (l''_k x_kj), with
// A-operand x (exact in BF16) and B-operand l''_k x_kj split into three BF16 terms
// (hi + mid + lo, residual below 2^-24 relative), so each product is as accurate as an FP32
// product. One CTA handles tiles of 128 rows: the rows are copied into shared memory in the
// MMA's canonical no-swizzle MN-major layout (16-byte cp.async units), one thread per row forms
// eta = x'theta and the family terms in FP64 (A, and l' for B), the same thread writes its row of
// the three B-operand tiles, one thread issues 3 x 8 MMAs (K = 16 each) and commits them to an
// mbarrier. Every kDrain tiles the FP32 accumulator is read back (tcgen05.ld) and added to FP64
// accumulators of the upper triangle in shared memory; B is accumulated in FP64 by column
// threads. Per-CTA partials use the layout of the SIMT moment kernel, so the same FP64 reduction
// (fixed order over blocks) finishes A, B and C.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "device.cuh"
#include "internal.h"

namespace subsmc {
namespace {

constexpr int kRows = 128;      // rows per tile = MMA M extent of the row operand = threads
constexpr int kM = 128;         // MMA M: covariate index i (p <= 128, zero-padded)
constexpr int kKGroups = kRows / 8;
constexpr int kStrip = kKGroups * 128;  // bytes of one 8-column strip of a tile (all 128 rows)
constexpr int kDrain = 4;       // tiles accumulated in FP32 in tensor memory between FP64 drains
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at the maximum SM clock

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor (tcgen05): start address, leading (K-direction) and stride
// (MN-direction) byte offsets between 8 x 16-byte core matrices, fixed bits 46-48 = 0b001, no
// swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor, kind::f16: FP32 accumulator, BF16 A and B, both MN-major, M x N.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
         ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      "selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void fence_barrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                   smem_u32(dst)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(taddr), "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void mma_bf16(uint32_t dtmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(dtmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
          smem_u32(bar))
      : "memory");
}
// 8 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float *v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[e]);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(smem)), "l"(gmem)
               : "memory");
}

// Round-to-nearest BF16 bits of an FP32 value, and the value of those bits.
__device__ __forceinline__ uint32_t bf16_bits(float v) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(v));
}
__device__ __forceinline__ float bf16_val(uint32_t b) { return __uint_as_float(b << 16); }

// Byte offset of unit (row k, 8-column strip c) in a tile: strips of kStrip bytes, 8-row core
// matrices of 128 bytes within a strip, 16 bytes per row.
__device__ __forceinline__ int unit_off(int k, int c) { return c * kStrip + (k >> 3) * 128 + (k & 7) * 16; }

template <int FAM>
__global__ void __launch_bounds__(kRows) k_cv_mma(const __nv_bfloat16 *Xp, int64_t n, int p, int S,
                                                  int Yo, double s2, double nu,
                                                  const double *theta, double *part, int N,
                                                  int ncols) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nvx = (p + 7) / 8;   // 16-byte units of covariates per row
  const int nb = N / 8;          // strips of the B operand
  const int np = p * (p + 1) / 2;
  // shared layout: A tile | 3 B tiles | theta | l' | C accumulators | reduction | mbarrier | taddr
  unsigned char *At = sm;
  unsigned char *Bt = At + kM / 8 * kStrip;
  double *ths = reinterpret_cast<double *>(Bt + 3 * nb * kStrip);
  double *lps = ths + 128;
  double *Cacc = lps + kRows;
  double *red = Cacc + ((np + 1) & ~1);
  uint64_t *bar = reinterpret_cast<uint64_t *>(red + 32);
  uint32_t *tptr = reinterpret_cast<uint32_t *>(bar + 1);

  for (int c = tid; c < 128; c += kRows) ths[c] = c < p ? theta[c] : 0.0;
  for (int q = tid; q < np; q += kRows) Cacc[q] = 0.0;
  // strips that no copy or write ever fills stay zero
  for (int off = tid * 16; off < kM / 8 * kStrip; off += kRows * 16)
    if (off / kStrip >= nvx) *reinterpret_cast<uint4 *>(At + off) = make_uint4(0u, 0u, 0u, 0u);
  for (int off = tid * 16; off < 3 * nb * kStrip; off += kRows * 16)
    if ((off / kStrip) % nb >= nvx) *reinterpret_cast<uint4 *>(Bt + off) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) tmem_alloc(tptr, (uint32_t)ncols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tptr;
  const uint32_t idesc = instr_desc(kM, N);
  const uint32_t a_base = smem_u32(At), b_base = smem_u32(Bt);

  double Aacc = 0.0, Bacc = 0.0;
  const int bgroups = kRows / p, bgrp = tid / p, bcol = tid - (tid / p) * p;
  uint32_t phase = 0;
  int since_drain = 0;
  bool timed_out = false;
  const int64_t ntiles = (n + kRows - 1) / kRows;
  for (int64_t tile = blockIdx.x; tile < ntiles && !timed_out; tile += gridDim.x) {
    const int64_t r0 = tile * kRows;
    // 1. the tile's covariates, MN-major (a unit = 8 consecutive columns of one row)
    for (int u = tid; u < kRows * nvx; u += kRows) {
      const int k = u / nvx, c = u - k * nvx;
      unsigned char *dst = At + unit_off(k, c);
      if (r0 + k < n)
        cp_async16(dst, Xp + (r0 + k) * S + 8 * c);
      else
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // 2. one thread per row: eta, the family terms (FP64), A; its row of the B-operand tiles
    {
      const int k = tid;
      const bool in = r0 + k < n;
      double l = 0.0, d1 = 0.0, d2 = 0.0;
      if (in) {
        double ep[8] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};  // independent FP64 chains
        for (int c = 0; c < nvx; ++c) {
          const uint4 w = *reinterpret_cast<const uint4 *>(At + unit_off(k, c));
          float x[8];
          Store<__nv_bfloat16>::unpack(w, x);
#pragma unroll
          for (int e = 0; e < 8; ++e) ep[e] = fma((double)x[e], ths[8 * c + e], ep[e]);
        }
        const double eta = ((ep[0] + ep[1]) + (ep[2] + ep[3])) + ((ep[4] + ep[5]) + (ep[6] + ep[7]));
        const RowC<float> *tl = reinterpret_cast<const RowC<float> *>(Xp + (r0 + k) * S + Yo);
        row_value<FAM>(eta, (double)__ldg(&tl->y), s2, nu, l, d1, d2);
      }
      Aacc += l;
      lps[k] = d1;
      const float wk = (float)d2;
      for (int c = 0; c < nvx; ++c) {
        const uint4 w = *reinterpret_cast<const uint4 *>(At + unit_off(k, c));
        float x[8];
        Store<__nv_bfloat16>::unpack(w, x);
        uint32_t hb[8], mb[8], lb[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const float v = wk * x[e];
          hb[e] = bf16_bits(v);
          const float r1 = v - bf16_val(hb[e]);
          mb[e] = bf16_bits(r1);
          lb[e] = bf16_bits(r1 - bf16_val(mb[e]));
        }
        const int off = unit_off(k, c);
        *reinterpret_cast<uint4 *>(Bt + off) =
            make_uint4(hb[0] | hb[1] << 16, hb[2] | hb[3] << 16, hb[4] | hb[5] << 16, hb[6] | hb[7] << 16);
        *reinterpret_cast<uint4 *>(Bt + nb * kStrip + off) =
            make_uint4(mb[0] | mb[1] << 16, mb[2] | mb[3] << 16, mb[4] | mb[5] << 16, mb[6] | mb[7] << 16);
        *reinterpret_cast<uint4 *>(Bt + 2 * nb * kStrip + off) =
            make_uint4(lb[0] | lb[1] << 16, lb[2] | lb[3] << 16, lb[4] | lb[5] << 16, lb[6] | lb[7] << 16);
      }
    }
    fence_proxy_async();  // this thread's generic-proxy writes become visible to the MMAs
    tc_fence_before();
    __syncthreads();
    // 3. B in FP64 (column threads) while one thread issues the MMAs
    if (tid == 0) {
      tc_fence_after();
#pragma unroll 1
      for (int q = 0; q < kRows / 16; ++q) {
        const uint64_t ad = smem_desc(a_base + q * 256, 128, kStrip);
#pragma unroll
        for (int s = 0; s < 3; ++s) {
          const uint64_t bd = smem_desc(b_base + s * nb * kStrip + q * 256, 128, kStrip);
          mma_bf16(tmem, ad, bd, idesc, (since_drain > 0 || q > 0 || s > 0) ? 1u : 0u);
        }
      }
      mma_commit(bar);
    }
    // B: thread (g, c) of the bgroups groups of p threads takes column c of rows g, g + bgroups,
    // .. (the FP64 work of a tile spread over all warps; the groups are merged once at the end)
    if (bgrp < bgroups) {
      const int c = bcol >> 3, e = bcol & 7;
      double b2[2] = {0.0, 0.0};  // independent FP64 chains
#pragma unroll 4
      for (int k = bgrp, t = 0; k < kRows; k += bgroups, ++t) {
        const float x = __bfloat162float(
            *reinterpret_cast<const __nv_bfloat16 *>(At + unit_off(k, c) + 2 * e));
        b2[t & 1] = fma(lps[k], (double)x, b2[t & 1]);
      }
      Bacc += b2[0] + b2[1];
    }
    // 4. wait for the MMAs (bounded in time; a timeout is reported as a NaN A partial)
    {
      const long long t0 = clock64();
      bool done = mbar_try_wait(bar, phase);
      while (!done && clock64() - t0 < kWaitCycles) done = mbar_try_wait(bar, phase);
      timed_out = __syncthreads_or(!done) != 0;
    }
    phase ^= 1u;
    tc_fence_after();
    ++since_drain;
    const bool last = tile + gridDim.x >= ntiles;
    // 5. drain the FP32 accumulator into the FP64 upper triangle
    if (!timed_out && (since_drain == kDrain || last)) {
      const int i = warp * 32 + lane;  // TMEM lane = covariate index i
      for (int j0 = 0; j0 < N; j0 += 8) {
        float v[8];
        tmem_ld8(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)j0, v);
        if (i < p) {
          const int rowoff = i * p - i * (i - 1) / 2 - i;  // index of (i, j) = rowoff + j, j >= i
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int j = j0 + e;
            if (j >= i && j < p) Cacc[rowoff + j] += (double)v[e];
          }
        }
      }
      since_drain = 0;
    }
    tc_fence_before();
    __syncthreads();  // the tile's shared memory and the accumulator may be reused
  }
  // partials: A, B, C (upper triangle, row-major), as the SIMT kernel writes them
  double *out = part + (int64_t)blockIdx.x * (1 + p + np);
  if (tid < 32) red[tid] = 0.0;
  __syncthreads();
  const double As = warp_sum(Aacc);
  if (lane == 0) red[warp] = As;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < kRows / 32; ++w) t += red[w];
    out[0] = timed_out ? __longlong_as_double(0x7FF8000000000000ll) : t;
  }
  lps[tid] = Bacc;  // the tiles are done with lps: it collects the groups' B partials
  __syncthreads();
  if (tid < p) {
    double b = 0.0;
    for (int g = 0; g < bgroups; ++g) b += lps[g * p + tid];
    out[1 + tid] = b;
  }
  for (int q = tid; q < np; q += kRows) out[1 + p + q] = Cacc[q];
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tmem, (uint32_t)ncols);
  }
}

// Tensor-memory columns for an N-column accumulator (a power of two, at least 32).
int tmem_cols(int N) {
  int c = 32;
  while (c < N) c <<= 1;
  return c;
}

size_t cv_mma_smem(int p, int N) {
  const int np = p * (p + 1) / 2;
  return (size_t)kM / 8 * kStrip + (size_t)3 * (N / 8) * kStrip +
         sizeof(double) * (128 + kRows + ((np + 1) & ~1) + 32) + 16;
}

template <int FAM>
int launch_fam(const __nv_bfloat16 *Xp, int64_t n, int p, int S, int Yo, double s2, double nu,
               const double *theta, double *part, int maxblocks, int *nblocks, cudaStream_t s) {
  const int N = ((p + 15) / 16) * 16;
  const size_t smem = cv_mma_smem(p, N);
  cudaError_t e = cudaFuncSetAttribute(k_cv_mma<FAM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return (int)e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cv_mma<FAM>, kRows, smem);
  if (e != cudaSuccess) return (int)e;
  if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int cols = tmem_cols(N);
  if (per_sm * cols > 512) per_sm = 512 / cols;  // every resident CTA gets its columns at once
  const int64_t ntiles = (n + kRows - 1) / kRows;
  int64_t grid = (int64_t)per_sm * sms;
  if (grid > maxblocks) grid = maxblocks;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  *nblocks = (int)grid;
  k_cv_mma<FAM><<<(int)grid, kRows, smem, s>>>(Xp, n, p, S, Yo, s2, nu, theta, part, N, cols);
  return (int)cudaGetLastError();
}

}  // namespace

// Partials of A, B, C for BF16 storage with p <= 128 on the tensor cores; writes the number of
// partial blocks used to *nblocks. Returns a cudaError_t (cudaErrorInvalidValue if p > 128).
int cv_moments_mma(const void *Xp, int64_t n, int p, int S, int Yo, int fam, double sigma2,
                   double nu, const double *theta, double *partials, int maxblocks, int *nblocks,
                   cudaStream_t s) {
  if (p < 1 || p > kM) return (int)cudaErrorInvalidValue;
  const __nv_bfloat16 *X = (const __nv_bfloat16 *)Xp;
  const double v = nu;
  switch (fam) {
    case 0: return launch_fam<0>(X, n, p, S, Yo, sigma2, v, theta, partials, maxblocks, nblocks, s);
    case 1: return launch_fam<1>(X, n, p, S, Yo, sigma2, v, theta, partials, maxblocks, nblocks, s);
    case 2: return launch_fam<2>(X, n, p, S, Yo, sigma2, v, theta, partials, maxblocks, nblocks, s);
    case 3: return launch_fam<3>(X, n, p, S, Yo, sigma2, v, theta, partials, maxblocks, nblocks, s);
    default: return launch_fam<4>(X, n, p, S, Yo, sigma2, v, theta, partials, maxblocks, nblocks, s);
  }
}

}  // namespace subsmc
