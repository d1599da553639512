// HMC trajectory with the particle's subsample resident in shared memory and both per-row
// contractions on the tensor cores (Algorithm 1 step 2; BF16 storage of X, p <= 32).
//
// An estimator pass at theta needs, for the particle's m gathered rows x_j,
//   D_j = x_j'(theta - theta_bar)                        (one dot product per row)
//   G1 = sum_j r_j x_j,  G2 = sum_j e_j r_j x_j          (two weighted column sums)
// with the per-row terms d_j, r_j of the family in between (device.cuh; e_j = d_j - K, the sums
// shifted as in the other estimator kernels). Both are contractions with the particle's own rows
// X_u [m x p], so per pass the CTA runs
//   GEMM1  D[j, n]  = sum_c X_u[j, c] Delta[c, n]     M = 128 rows per tile, N = 16, K = 32
//   GEMM2  G[c, n]  = sum_j X_u[j, c] Q[j, n]         M = 128 (columns c), N = 16, K = m
// with tcgen05.mma (kind::f16, BF16 operands, FP32 accumulators in tensor memory). X is exact in
// BF16. delta = theta - theta_bar enters as three BF16 terms (columns 0..2 of Delta: hi, middle,
// low; their sum carries 24 bits), so D keeps FP32 accuracy; r_j and e_j r_j enter the same way
// (Q columns 0, 2, 4 and 1, 3, 5). The CUDA cores are left with the row terms: read D from tensor
// memory, evaluate d_j, r_j, split r_j and e_j r_j into BF16 terms and store one 16-byte row of Q.
//
// Shared memory holds X_u once, in 8-row groups of nq = ceil(p/8) core matrices of 8 rows x 8
// columns (16 bytes per row): row j, columns 8q..8q+7 at (j/8) nq 128 + q 128 + (j%8) 16. The same
// bytes are the K-major A operand of GEMM1 (core stride 128 along K = columns, nq 128 along M =
// rows) and the MN-major A operand of GEMM2 (nq 128 along K = rows, 128 along M = columns). The
// tensor core reads past the nq real chunks of a group where an MMA is wider than p: in GEMM1 it
// multiplies them by the zero rows of Delta (columns >= p), in GEMM2 they land in accumulator rows
// c >= 8 nq that are never read; a zero-filled guard after the rows keeps every such read inside
// the CTA's allocation.
//
// One CTA (8 warps) per particle, persistent over particles. Warp w reads tensor-memory lane
// quadrant w % 4 (rows 128 t + 32 (w % 4) + lane) of the tiles t = w / 4, w / 4 + 2, ...; warp 0
// also carries theta, rho and the gradient one column per lane and runs the leapfrog and the FP64
// Hamiltonian; thread 0 issues the MMAs. Every mbarrier wait is bounded; on a timeout the kernel
// raises the iteration-cap error bit and returns after freeing its tensor memory.
#pragma once

#include "resident.cuh"

namespace subsmc {
namespace tc {

constexpr int kWarps = 8;
constexpr int kThreads = kWarps * 32;
constexpr int kN = 16;               // MMA N of both GEMMs (M = 128 needs N a multiple of 16)
constexpr int kTmemCols = 256;       // GEMM1 tiles use 16 columns each (<= 15 tiles), GEMM2 16
constexpr int kMaxTiles = 15;        // m <= 1920
constexpr long long kWaitCycles = 2000000000ll;
constexpr int kMinSmem = 80 * 1024;  // at most two CTAs per SM: 2 x 256 tensor-memory columns

__device__ __forceinline__ uint32_t su32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
// No-swizzle shared-memory matrix descriptor: LBO = byte stride between core matrices adjacent
// along K, SBO = along M or N; bits 46-48 = 0b001 (the same convention as the full-data kernel).
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B; a_mn / b_mn: MN-major operand.
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
// Bounded wait of the whole CTA on an mbarrier phase; gives up early when *abort is set (by the
// warp whose own wait timed out). False on every thread if any thread gave up.
__device__ __forceinline__ bool cta_wait(uint64_t *bar, uint32_t parity, volatile int *abort) {
  const long long t0 = clock64();
  bool done = try_wait(bar, parity);
  while (!done && *abort == 0 && clock64() - t0 < kWaitCycles) done = try_wait(bar, parity);
  return __syncthreads_and(done) != 0;
}
// Bounded wait of one warp.
__device__ __forceinline__ bool warp_wait(uint64_t *bar, uint32_t parity) {
  const long long t0 = clock64();
  bool done = try_wait(bar, parity);
  while (!done && clock64() - t0 < kWaitCycles) done = try_wait(bar, parity);
  return __all_sync(0xffffffffu, done) != 0;
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
// Columns col .. col+3 of this thread's tensor-memory lane (no wait).
__device__ __forceinline__ void ld4(uint32_t taddr, uint32_t *r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
}
__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t *r) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr));
}
__device__ __forceinline__ void ld_wait() {
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}
__device__ __forceinline__ uint32_t pack_bf2(float lo, float hi) {
  const __nv_bfloat162 b = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<const uint32_t *>(&b);
}
__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// Shared-memory plan of one CTA (byte offsets).
struct TcPlan {
  int nq, mpad, ntile;
  int off_rc, off_q, off_dl, off_dv, off_rd, off_blk, off_rho0, off_bar, off_misc, total;
};

inline TcPlan tc_plan(int p, int m, int G) {
  TcPlan P;
  P.nq = (p + 7) / 8;
  P.mpad = ((m + 127) / 128) * 128;
  P.ntile = P.mpad / 128;
  int off = P.mpad * P.nq * 16 + 2048;  // rows and the guard the MMAs may read past them
  P.off_rc = off;                       // row constants (tails) [mpad]
  off += P.mpad * 16;
  P.off_q = off;                        // Q: [mpad/8 groups][2 N halves][8 rows][16 B]
  off += P.mpad * 32;
  P.off_dl = off;                       // Delta: [4 K chunks][2 N halves][8][16 B]
  off += 4 * 256;
  P.off_dv = off;                       // e_j of the last pass (block sums) [m]
  off += ((m * 4 + 15) / 16) * 16;
  P.off_rd = off;                       // per-warp sums of e, e^2 [kWarps][2] (state type)
  off += kWarps * 2 * 4;
  off = (off + 15) & ~15;
  P.off_blk = off;                      // block sums [G][2] double
  off += G * 2 * 8;
  P.off_rho0 = off;                     // C and Sigma, zero-padded to [32][32] float each
  off += 2 * 32 * 32 * 4;
  P.off_bar = off;                      // two mbarriers, tensor-memory address, abort flag
  off += 32;
  P.off_misc = off;
  off += 16;
  P.total = off < kMinSmem ? kMinSmem : off;
  return P;
}

template <int F>
__device__ __forceinline__ void tc_row(const RowC<float> &c, float D, float inv_s2, float K,
                                       int cv1, float &e, float &r) {
  float d;
  row_incr<F, float>(c, D, inv_s2, d, r);
  if (cv1) to_first_order(row_l2<F, float>(c, inv_s2), D, d, r);
  e = d - K;
}

__global__ void __launch_bounds__(kThreads, 2) k_hmc_tc(EstArgs a, TcPlan P) {
  extern __shared__ __align__(128) unsigned char sm[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int quad = warp & 3, half = warp >> 2;
  const int p = a.p, m = a.m, G = a.G, S = a.S, nq = P.nq;
  const __nv_bfloat16 *Xp = reinterpret_cast<const __nv_bfloat16 *>(a.Xp);
  unsigned char *Xs = sm;
  RowC<float> *Rc = reinterpret_cast<RowC<float> *>(sm + P.off_rc);
  unsigned char *Qs = sm + P.off_q;
  unsigned char *Ds = sm + P.off_dl;
  float *dv = reinterpret_cast<float *>(sm + P.off_dv);
  float *rd = reinterpret_cast<float *>(sm + P.off_rd);
  double *blks = reinterpret_cast<double *>(sm + P.off_blk);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + P.off_bar);
  uint32_t *tptr = reinterpret_cast<uint32_t *>(bar + 2);
  volatile int *abort = reinterpret_cast<volatile int *>(bar + 2) + 1;

  // zero everything once: guard, padding rows, the unused halves of Q and Delta stay zero
  for (int o = tid * 16; o < P.off_bar; o += kThreads * 16)
    *reinterpret_cast<uint4 *>(sm + o) = make_uint4(0u, 0u, 0u, 0u);
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar)) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(su32(bar + 1)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    *abort = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     su32(tptr)),
                 "n"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tptr;
  const uint32_t tG = tmem + 16 * kMaxTiles;                // GEMM2 accumulator columns
  const uint32_t tq = tmem + ((uint32_t)(quad * 32) << 16);  // this warp's lane quadrant
  const uint32_t id1 = idesc(128, kN, 0, 0), id2 = idesc(128, kN, 1, 1);
  const uint32_t xsb = su32(Xs), qb = su32(Qs), db = su32(Ds);
  uint32_t phA = 0, phB = 0;
  bool ok = true;

  const double temp = a.st->a;
  const float inv_s2 = (float)a.inv_s2;
  const double nm = (double)a.n / (double)m, inv_m = 1.0 / (double)m;
  const float ta = (float)temp, ta2 = (float)(temp * temp * nm * nm), tnm = (float)(temp * nm);
  const uint32_t smv = stage_move(a.stage_dev ? a.st->stage : a.stage, a.move);
  const int fam = a.fam;
  const int cv1 = a.cv_order == 1;
  const bool col = lane < p;
  const float Bc = col ? ldg_ct<float>(a.B_ct, lane) : 0.f;
  const float muc = col ? ldg_ct<float>(a.mu_ct, lane) : 0.f;
  const float ivc = col ? ldg_ct<float>(a.ivar_ct, lane) : 0.f;
  const float tbc = col ? ldg_ct<float>(a.tb_ct, lane) : 0.f;
  float *Cs = reinterpret_cast<float *>(sm + P.off_rho0);  // [32][32], C[k][c] at k * 32 + c
  float *Ss = Cs + 32 * 32;                                 // Sigma, the same layout
  for (int e = tid; e < 32 * 32; e += kThreads) {
    const int r = e >> 5, c = e & 31;
    const bool in = r < p && c < p;
    Cs[e] = in ? ldg_ct<float>(a.C_ct, r * p + c) : 0.f;
    Ss[e] = in ? ldg_ct<float>(a.Sigma_ct, r * p + c) : 0.f;
  }
  __syncthreads();
  // (M v)_lane for a symmetric [32][32] matrix in shared memory and v one column per lane
  auto matvec = [&](const float *M, float v) -> float {
    float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
    for (int k = 0; k < 32; k += 2) {
      acc0 = fmaf(M[k * 32 + lane], __shfl_sync(0xffffffffu, v, k), acc0);
      acc1 = fmaf(M[(k + 1) * 32 + lane], __shfl_sync(0xffffffffu, v, k + 1), acc1);
    }
    return acc0 + acc1;
  };

  // Descriptors advance by adding to their start-address field ((address >> 4) in bits 0-13;
  // every address here is below 256 KB, so the field never carries into the next one).
  const uint64_t a1 = desc(xsb, 128, nq * 128), b1 = desc(db, 256, 128);
  const uint64_t a2 = desc(xsb, nq * 128, 128), b2 = desc(qb, 256, 128);
  const uint64_t a1_tile = (uint64_t)(16 * nq * 128) >> 4, a2_step = (uint64_t)(2 * nq * 128) >> 4;
  // GEMM1 for the delta now in Delta (thread 0): every row tile, K = 32 in two steps
  auto issue_gemm1 = [&]() {
    fence_after();
    uint64_t ad = a1;
    for (int t = 0; t < P.ntile; ++t, ad += a1_tile) {
      mma(tmem + 16 * t, ad, b1, id1, 0u);
      mma(tmem + 16 * t, ad + (256 >> 4), b1 + (512 >> 4), id1, 1u);
    }
    commit(bar);
  };
  // GEMM2 for the rows' Q now in shared memory (thread 0): K = mpad in steps of 16 rows
  auto issue_gemm2 = [&]() {
    fence_after();
    uint64_t ad = a2, bd = b2;
    const int nk = P.mpad / 16;
    mma(tG, ad, bd, id2, 0u);
    for (int s = 1; s < nk; ++s) {
      ad += a2_step;
      bd += (512 >> 4);
      mma(tG, ad, bd, id2, 1u);
    }
    commit(bar + 1);
  };
  // delta in Delta: column c, terms hi / middle / low at N = 0, 1, 2 (warp 0, all lanes)
  auto write_delta = [&](float th) {
    if (lane < 32) {
      const float dl = col ? th - tbc : 0.f;
      const __nv_bfloat16 h = __float2bfloat16_rn(dl);
      const float r1 = dl - __bfloat162float(h);
      const __nv_bfloat16 mdl = __float2bfloat16_rn(r1);
      const __nv_bfloat16 lo = __float2bfloat16_rn(r1 - __bfloat162float(mdl));
      unsigned char *base = Ds + (lane >> 3) * 256 + (lane & 7) * 2;
      *reinterpret_cast<__nv_bfloat16 *>(base) = h;
      *reinterpret_cast<__nv_bfloat16 *>(base + 16) = mdl;
      *reinterpret_cast<__nv_bfloat16 *>(base + 32) = lo;
    }
    fence_async();
    __syncwarp();
  };

  for (int il = blockIdx.x; il < a.B && ok; il += gridDim.x) {
    const int i = a.i0 + il;  // global particle index
    const int32_t *u = a.u + (int64_t)i * m;
    __syncthreads();  // the previous particle is finished with shared and tensor memory
    // 1. gather the rows (covariate chunks and tails) with 16-byte copies; bad indices flagged,
    // their rows zeroed. The indices are staged in shared memory first (dv is free until the last
    // pass), so no copy waits on a global load.
    int32_t *us = reinterpret_cast<int32_t *>(dv);
    for (int j = tid; j < m; j += kThreads) cp_async4(us + j, u + j);
    cp_async_wait_all();
    __syncthreads();
    const int nvr = nq + 1;
    for (int t = tid; t < m * nvr; t += kThreads) {
      const int j = t / nvr, q = t - j * nvr;
      const int k = us[j];
      unsigned char *dst = q < nq ? Xs + (j >> 3) * nq * 128 + q * 128 + (j & 7) * 16
                                  : reinterpret_cast<unsigned char *>(Rc + j);
      if (k < 0 || (int64_t)k >= a.n) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        if (q == 0) set_err(a.st, kErrIndex);
        continue;
      }
      const unsigned char *row = reinterpret_cast<const unsigned char *>(Xp + (int64_t)k * S);
      cp_async16(dst, q < nq ? row + 16 * q : row + a.Yo * 2);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
    fence_async();
    // 2. warp 0: momentum, theta, the shift of the sums from the cache, delta, GEMM1
    float *thg = reinterpret_cast<float *>(a.theta_out) + (int64_t)i * p;
    const float eps = (float)jittered_eps(a.st->eps, a.eps_jitter, a.seed, smv, (uint32_t)i);
    float th = 0.f, rho = 0.f, gr = 0.f;
    float Ksh = 0.f;
    if (a.blk) {
      const double *bc = a.blk + (int64_t)i * G * 2;
      double s0 = 0.0;
      for (int g = lane; g < G; g += 32) s0 += bc[2 * g];
      Ksh = (float)(warp_sum(s0) * inv_m);
      if (!isfinite(Ksh)) Ksh = 0.f;
    }
    if (warp == 0) {
      const Stream smom(a.seed, kMomentum, smv, (uint32_t)i);
      const float z = col ? (float)stream_normal(smom, (uint32_t)lane) : 0.f;
      float acc = 0.f;
      for (int c = 0; c < p; ++c) {  // rho_r = sum_{c >= r} Linv[c, r] z_c
        const float zc = __shfl_sync(0xffffffffu, z, c);
        if (col && c >= lane) acc = fmaf(ldg_ct<float>(a.Linv_ct, c * p + lane), zc, acc);
      }
      rho = col ? acc : 0.f;
      th = col ? thg[lane] : 0.f;
      write_delta(th);
    }
    fence_before();
    __syncthreads();  // rows, tails and Delta are in shared memory
    if (tid == 0) issue_gemm1();

    auto kinetic = [&]() -> double {  // rho' Sigma rho / 2 (warp 0)
      const float v = matvec(Ss, rho);
      return 0.5 * warp_sum(col ? (double)rho * (double)v : 0.0);
    };
    auto log_prior = [&]() -> double {
      const double rr = (double)th - (double)muc;
      return warp_sum(col ? -0.5 * rr * rr * (double)ivc : 0.0) + a.log_prior_const;
    };
    double ell = 0.0, sig = 0.0, H0 = 0.0;
    double kin0 = 0.0, lp0 = 0.0;
    if (warp == 0) {
      kin0 = kinetic();
      lp0 = log_prior();
    }

    // 3. the L + 1 estimator passes. A failed wait of warp 0 sets *abort and bad0; the other
    // warps then leave at their next CTA-wide wait, so every exit from the loop is uniform.
    bool bad0 = false;
    for (int l = 0; l <= a.L; ++l) {
      const bool final = l == a.L, totals = l == 0 || final;
      if (!cta_wait(bar, phA, abort)) {
        ok = false;
        break;
      }
      phA ^= 1u;
      fence_after();
      // rows of this warp: tiles t = half, half + 2, ...; row j = 128 t + 32 quad + lane
      float sd = 0.f, sd2 = 0.f;
      // D of every tile of this warp first (one wait for all the tensor-memory loads)
      uint32_t vt[(kMaxTiles + 1) / 2][4];
#pragma unroll
      for (int k = 0; k < (kMaxTiles + 1) / 2; ++k)
        if (half + 2 * k < P.ntile) ld4(tq + 16 * (half + 2 * k), vt[k]);
      ld_wait();
      auto rows = [&](auto famc) {
        constexpr int F = decltype(famc)::value;
#pragma unroll
        for (int k = 0; k < (kMaxTiles + 1) / 2; ++k) {
          const int t = half + 2 * k;
          if (t >= P.ntile) break;
          const uint32_t *v = vt[k];
          const int j = 128 * t + 32 * quad + lane;
          if (j < m) {
            const float D = __uint_as_float(v[0]) + __uint_as_float(v[1]) + __uint_as_float(v[2]);
            float e, r;
            tc_row<F>(Rc[j], D, inv_s2, Ksh, cv1, e, r);
            sd += e;
            sd2 = fmaf(e, e, sd2);
            if (final) dv[j] = e;
            const float er = e * r;
            const uint32_t h = pack_bf2(r, er);
            const float r1 = r - bf_lo(h), q1 = er - bf_hi(h);
            const uint32_t md = pack_bf2(r1, q1);
            const uint32_t lo = pack_bf2(r1 - bf_lo(md), q1 - bf_hi(md));
            *reinterpret_cast<uint4 *>(Qs + (j >> 3) * 256 + (j & 7) * 16) =
                make_uint4(h, md, lo, 0u);
          }
        }
      };
      switch (fam) {
        case 0: rows(std::integral_constant<int, 0>{}); break;
        case 1: rows(std::integral_constant<int, 1>{}); break;
        case 2: rows(std::integral_constant<int, 2>{}); break;
        case 3: rows(std::integral_constant<int, 3>{}); break;
        default: rows(std::integral_constant<int, 4>{}); break;
      }
      const float s1 = warp_sum(sd), s2 = warp_sum(sd2);
      if (lane == 0) {
        rd[2 * warp] = s1;
        rd[2 * warp + 1] = s2;
      }
      fence_async();
      fence_before();
      __syncthreads();  // Q complete, all reads of GEMM1's accumulators done
      if (tid == 0) issue_gemm2();
      float S1f = 0.f;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) S1f += rd[2 * w];
      const float ebar = S1f * (float)inv_m;  // mean of e this pass
      if (final) {  // shifted block sums of e (floor partition of u into G blocks)
        for (int g = warp; g < G; g += kWarps) {
          const int j0 = (int)(((int64_t)g * m) / G), j1 = (int)(((int64_t)(g + 1) * m) / G);
          float bs = 0.f, bq = 0.f;
          for (int j = j0 + lane; j < j1; j += 32) {
            const float dj = dv[j];
            bs += dj;
            bq = fmaf(dj, dj, bq);
          }
          bs = warp_sum(bs);
          bq = warp_sum(bq);
          if (lane == 0) {
            blks[2 * g] = (double)bs;
            blks[2 * g + 1] = (double)bq;
          }
        }
        __syncthreads();
      }
      if (warp == 0 && !bad0) {
        // 4. the gradient from GEMM2, the totals, the leapfrog
        if (!warp_wait(bar + 1, phB)) {
          *abort = 1;
          bad0 = true;
        } else {
          fence_after();
          uint32_t g8[8];
          ld8(tG, g8);
          ld_wait();
          const float G1 = __uint_as_float(g8[0]) + __uint_as_float(g8[2]) + __uint_as_float(g8[4]);
          const float G2 = __uint_as_float(g8[1]) + __uint_as_float(g8[3]) + __uint_as_float(g8[5]);
          const float dl = col ? th - tbc : 0.f;
          const float cd = matvec(Cs, dl);  // (C delta)_c
          gr = col ? ta * (Bc + cd) + tnm * G1 - ta2 * (G2 - ebar * G1) - (th - muc) * ivc : 0.f;
          if (totals) {  // l_hat and sigma2_hat in FP64 (first and last pass)
            const float qlin = warp_sum(col ? dl * (Bc + 0.5f * cd) : 0.f);
            double S1 = 0.0, S2 = 0.0;
            if (final) {
              for (int g = 0; g < G; ++g) {
                S1 += blks[2 * g];
                S2 += blks[2 * g + 1];
              }
            } else {
              for (int w = 0; w < kWarps; ++w) {
                S1 += (double)rd[2 * w];
                S2 += (double)rd[2 * w + 1];
              }
            }
            ell = (a.A_dev ? __ldg(a.A_dev) : a.A) + (double)qlin +
                  nm * fma((double)m, (double)Ksh, S1);
            sig = nm * nm * fmax(0.0, S2 - S1 * S1 * inv_m);
          }
          if (l == 0) H0 = -(temp * ell - 0.5 * temp * temp * sig + lp0) + kin0;
          if (l > 0) rho += 0.5f * eps * gr;  // closing half-kick of step l
          if (!final) {
            rho += 0.5f * eps * gr;  // opening half-kick of step l + 1
            const float vs = matvec(Ss, rho);  // (Sigma rho)_c
            if (col) th += eps * vs;
            write_delta(th);
            fence_before();
            if (lane == 0) issue_gemm1();
          }
        }
      }
      phB ^= 1u;
      if (!final) Ksh += ebar;  // the next pass is shifted by this pass's mean of d
      if (final && !__syncthreads_and(!bad0)) ok = false;  // warp 0's last wait, made uniform
    }
    if (!ok) break;
    // 5. Metropolis-Hastings in FP64, write-back on acceptance (warp 0)
    if (warp == 0) {
      const double kin1 = kinetic(), lp1 = log_prior();
      const double H1 = -(temp * ell - 0.5 * temp * temp * sig + lp1) + kin1;
      const Stream smh(a.seed, kMhTheta, smv, (uint32_t)i);
      const double Uu = draw_uniform(smh.draw(0));
      const bool acc = log(Uu) < H0 - H1;  // false when H1 is NaN
      if (acc) {
        if (col) thg[lane] = th;
        double *blk = a.blk + (int64_t)i * G * 2;
        const double k = (double)Ksh;
        for (int g = lane; g < G; g += 32) {
          const double ng = (double)((int)(((int64_t)(g + 1) * m) / G) - (int)(((int64_t)g * m) / G));
          const double se = blks[2 * g], qe = blks[2 * g + 1];
          blk[2 * g] = fma(ng, k, se);
          blk[2 * g + 1] = qe + k * fma(ng, k, 2.0 * se);
        }
        if (lane == 0) {
          a.ell[i] = ell;
          a.sig2[i] = sig;
          atomicAdd(&a.st->acc_theta, 1ull);
        }
      }
    }
  }
  if (!ok && tid == 0) set_err(a.st, kErrCap);
  asm volatile("cp.async.wait_all;\n" ::: "memory");
  fence_before();
  __syncthreads();
  if (warp == 0) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                 "n"(kTmemCols)
                 : "memory");
  }
}

}  // namespace tc

// Launch of the tensor-core trajectory kernel (BF16 storage). dry: check the fit only. Returns a
// cudaError_t, or -2 when p > 32, m > 1920 or the shared-memory plan does not fit.
inline int launch_res_tc(const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  if (a.p > 32 || a.m > 128 * tc::kMaxTiles || a.m < 1) return -2;
  const tc::TcPlan P = tc::tc_plan(a.p, a.m, a.G);
  cudaError_t e = cudaFuncSetAttribute(tc::k_hmc_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       P.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  cudaFuncSetAttribute(tc::k_hmc_tc, cudaFuncAttributePreferredSharedMemoryCarveout,
                       (int)cudaSharedmemCarveoutMaxShared);
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, tc::k_hmc_tc, tc::kThreads, P.total);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return -2;
  }
  // CTAs per SM by shared memory alone (the occupancy query can answer for a smaller carveout);
  // registers allow two (launch bounds), and two CTAs of 256 tensor-memory columns fill an SM
  int dev = 0, smem_sm = 0, reserved = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  cudaDeviceGetAttribute(&reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev);
  const int by_smem = smem_sm / (P.total + reserved);
  if (by_smem > per_sm) per_sm = by_smem;
  if (per_sm > 2) per_sm = 2;
  if (dry || a.B <= 0) return 0;
  const int grid = a.B < per_sm * sms ? a.B : per_sm * sms;
  tc::k_hmc_tc<<<grid, tc::kThreads, P.total, s>>>(a, P);
  return (int)cudaGetLastError();
}

}  // namespace subsmc
