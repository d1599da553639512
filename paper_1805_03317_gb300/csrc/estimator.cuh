// Warp-per-particle subsampled estimator and the kernels built on it.
//
// One warp owns one particle. Its m subsampled rows are gathered straight from the packed row
// copy of the data: T lanes share a row and each lane reads CPL element slots with 128-bit loads,
// so a warp has 32/T rows in flight per step (times U for the unrolled variants). Per row the
// lanes form eta_bar = x'theta_bar and D = x'(theta - theta_bar) with an intra-group shuffle
// reduction, evaluate the increment-form terms d and r (device.cuh), and accumulate
//   sum d, sum d^2                 (per block of u when the block cache is refreshed)
//   sum r x, sum d r x             (gradient partials, kept in registers)
// which give (Sec. 3.2, Eq. difference_estimator_logl)
//   l_hat      = A + B'delta + delta'C delta/2 + (n/m) sum d
//   sigma2_hat = (n^2/m^2) (sum d^2 - (sum d)^2/m)
//   grad       = a (B + C delta + (n/m) sum r x) - a^2 (n^2/m^2)(sum d r x - dbar sum r x) - (theta-mu)/v
// The last line is the exact gradient of a*l_hat - a^2/2*sigma2_hat + log p(theta) for fixed u.
#pragma once

#include "device.cuh"
#include "internal.h"

namespace subsmc {

__device__ __forceinline__ void set_err(DevState *st, int bit) {
  if (st) atomicOr(&st->err, bit);
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Streamed rows. T lanes share a row and each holds CPL element slots of it (slot s of the lane
// is element gl*CPL + s of the packed row). Rows reach the lanes through a per-warp ring of NST
// stages in shared memory filled with 16-byte cp.async copies: while stage `step` is consumed the
// copies of stage step + NST - 1 are in flight. Each lane copies and later reads only its own
// chunk, so the ring needs no barriers, only the lane's own cp.async group accounting.
template <typename XT, int T, int CPL, int NST>
struct WarpEval {
  using SD = Store<XT>;
  using CT = typename SD::CT;
  using YT = typename SD::YT;
  static constexpr int RPW = 32 / T;                 // rows per warp per step
  static constexpr int NV = CPL / SD::VEC;           // 16-byte vectors per lane per row
  static constexpr int LB = CPL * (int)sizeof(XT);   // bytes per lane per row
  // lane stride in the ring: an odd multiple of 16 bytes, so 128-bit accesses of 8 consecutive
  // lanes fall in distinct bank groups
  static constexpr int LS = (LB / 16) % 2 ? LB : LB + 16;
  static constexpr int RING = NST * 32 * LS;         // ring bytes per warp
  static_assert(CPL % SD::VEC == 0, "CPL must be a whole number of 16-byte vectors");
  static_assert(T >= 1 && T <= 32 && (T & (T - 1)) == 0, "T must be a power of two");
  static_assert(NST >= 2, "at least double buffering");

  CT tb[CPL], dl[CPL];
  int lane, gl, rs;
  unsigned char *mine;  // this lane's chunk of stage 0 of the ring
  int ylane, yoff;      // the lane of a row group that holds y, and y's byte offset in its chunk

  // ring: this warp's RING bytes (16-byte aligned). Yo: element at which y starts its own
  // 16-byte vector in the packed row (the covariates occupy the vectors before it).
  __device__ __forceinline__ void init(unsigned char *ring, int Yo) {
    lane = threadIdx.x & 31;
    gl = lane & (T - 1);
    rs = lane / T;
    mine = ring + lane * LS;
    ylane = Yo / CPL;
    yoff = (Yo - ylane * CPL) * (int)sizeof(XT);
  }
  // Slot s of this lane is element (column) gl*CPL + s of a packed row.
  __device__ __forceinline__ void load_slots(const CT *vec, int p, CT *dst) const {
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
      const int c = gl * CPL + s;
      dst[s] = c < p ? vec[c] : CT(0);
    }
  }

  // Rows [j0, j1) of the index list idx. Accumulates gradient partials into g1, g2 (if GRAD)
  // and returns this lane's partial sums of d and d^2 (nonzero only on group leaders).
  template <bool GRAD>
  __device__ __forceinline__ void rows(const XT *__restrict__ Xp, int S, int Yo, int p, int64_t n,
                                       const int32_t *idx, int j0, int j1, int fam,
                                       CT inv_s2, CT *g1, CT *g2, CT &sd, CT &sd2,
                                       DevState *st) const {
    const int nsteps = (j1 - j0 + RPW - 1) / RPW;
    auto issue = [&](int step) {
      if (step < nsteps) {
        const int j = j0 + step * RPW + rs;
        unsigned char *dst = mine + (step % NST) * 32 * LS;
        bool ok = j < j1;
        const int k = ok ? idx[j] : 0;  // plain load: u-update indices are written by this warp
        if (ok && (k < 0 || (int64_t)k >= n)) {
          set_err(st, kErrIndex);
          ok = false;
        }
        const unsigned char *src =
            reinterpret_cast<const unsigned char *>(Xp + (int64_t)k * S) + gl * LB;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
          if (gl * CPL + v * SD::VEC > Yo) continue;  // vectors past the y vector are not read
          if (ok)
            cp_async16(dst + 16 * v, src + 16 * v);
          else
            *reinterpret_cast<uint4 *>(dst + 16 * v) = make_uint4(0u, 0u, 0u, 0u);
        }
      }
      cp_async_commit();  // one group per step (empty past the end) keeps the counting uniform
    };
#pragma unroll
    for (int q = 0; q < NST - 1; ++q) issue(q);
    for (int step = 0; step < nsteps; ++step) {
      issue(step + NST - 1);
      cp_async_wait<NST - 1>();  // this lane's copies of `step` have landed
      const unsigned char *src = mine + (step % NST) * 32 * LS;
      CT xv[CPL];
#pragma unroll
      for (int v = 0; v < NV; ++v) {  // covariate vectors only; the y vector and beyond are zero
        if (gl * CPL + v * SD::VEC < Yo) {
          SD::unpack(*reinterpret_cast<const uint4 *>(src + 16 * v), &xv[v * SD::VEC]);
        } else {
#pragma unroll
          for (int e = 0; e < SD::VEC; ++e) xv[v * SD::VEC + e] = CT(0);
        }
      }
      YT yl = YT(0);
      if (gl == ylane) yl = *reinterpret_cast<const YT *>(src + yoff);
      CT pe = CT(0), pd = CT(0);
#pragma unroll
      for (int s = 0; s < CPL; ++s) {
        pe = fma(xv[s], tb[s], pe);
        pd = fma(xv[s], dl[s], pd);
      }
#pragma unroll
      for (int o = T / 2; o; o >>= 1) {
        pe += __shfl_xor_sync(0xffffffffu, pe, o);
        pd += __shfl_xor_sync(0xffffffffu, pd, o);
      }
      const CT y = (CT)__shfl_sync(0xffffffffu, yl, (lane & ~(T - 1)) + ylane);
      CT d, r;
      switch (fam) {
        case 0: row_terms<0, CT>(pe, pd, y, inv_s2, d, r); break;
        case 1: row_terms<1, CT>(pe, pd, y, inv_s2, d, r); break;
        case 2: row_terms<2, CT>(pe, pd, y, inv_s2, d, r); break;
        default: row_terms<3, CT>(pe, pd, y, inv_s2, d, r); break;
      }
      if (j0 + step * RPW + rs >= j1) {
        d = CT(0);
        r = CT(0);
      }
      if (GRAD) {
        const CT dr = d * r;
#pragma unroll
        for (int s = 0; s < CPL; ++s) {
          g1[s] = fma(r, xv[s], g1[s]);
          g2[s] = fma(dr, xv[s], g2[s]);
        }
      }
      if (gl == 0) {
        sd += d;
        sd2 = fma(d, d, sd2);
      }
    }
    cp_async_wait<0>();
  }
};

// Shared-memory scratch of one warp: theta, delta, rho, grad, v [p each] and the reduced gradient
// partials G1, G2 [T*CPL each], all in the state type.
template <typename CT> struct WarpSmem {
  CT *th, *dl, *rho, *g, *v, *G1, *G2;
  __device__ __forceinline__ WarpSmem(CT *base, int p, int slots) {
    th = base;
    dl = th + p;
    rho = dl + p;
    g = rho + p;
    v = g + p;
    G1 = v + p;
    G2 = G1 + slots;
  }
  static __host__ __device__ int count(int p, int slots) { return 5 * p + 2 * slots; }
};

// Bytes of dynamic shared memory per warp: the row ring, then the WarpSmem arrays.
template <typename XT, int T, int CPL, int NST>
__host__ __device__ inline int warp_smem_bytes(int p) {
  using CT = typename Store<XT>::CT;
  const int b = WarpEval<XT, T, CPL, NST>::RING + WarpSmem<CT>::count(p, T * CPL) * (int)sizeof(CT);
  return (b + 15) & ~15;
}

template <typename CT> __device__ __forceinline__ CT ldg_ct(const void *p, int i) {
  return __ldg(reinterpret_cast<const CT *>(p) + i);
}

// One evaluation of the estimator for the warp's particle at theta (in sm.th / sm.dl).
// Reads rows of idx[0..m); GRAD: writes the target gradient to sm.g; BLOCKS: writes per-block
// (sum d, sum d^2) to blk_out[G*2]. Returns l_hat and sigma2_hat on every lane.
template <typename XT, int T, int CPL, int U, bool GRAD, bool BLOCKS>
__device__ __forceinline__ void eval_particle(const WarpEval<XT, T, CPL, U> &W, const EstArgs &a,
                                              const int32_t *idx, WarpSmem<typename Store<XT>::CT> &sm,
                                              double temp, double *blk_out, double &ell,
                                              double &sig2) {
  using CT = typename Store<XT>::CT;
  const XT *Xp = reinterpret_cast<const XT *>(a.Xp);
  const CT inv_s2 = (CT)a.inv_s2;
  CT g1[CPL], g2[CPL];
#pragma unroll
  for (int s = 0; s < CPL; ++s) g1[s] = g2[s] = CT(0);
  double S = 0.0, Q = 0.0;
  if (BLOCKS) {
    for (int g = 0; g < a.G; ++g) {
      const int j0 = (int)(((int64_t)g * a.m) / a.G), j1 = (int)(((int64_t)(g + 1) * a.m) / a.G);
      CT sd = CT(0), sd2 = CT(0);
      W.template rows<GRAD>(Xp, a.S, a.Yo, a.p, a.n, idx, j0, j1, a.fam, inv_s2, g1, g2, sd, sd2, a.st);
      const double bs = warp_sum((double)sd), bq = warp_sum((double)sd2);
      if (W.lane == 0) {
        blk_out[2 * g] = bs;
        blk_out[2 * g + 1] = bq;
      }
      S += bs;
      Q += bq;
    }
  } else {
    CT sd = CT(0), sd2 = CT(0);
    W.template rows<GRAD>(Xp, a.S, a.Yo, a.p, a.n, idx, 0, a.m, a.fam, inv_s2, g1, g2, sd, sd2, a.st);
    S = warp_sum((double)sd);
    Q = warp_sum((double)sd2);
  }
  const double nm = (double)a.n / (double)a.m;
  const double dbar = S / (double)a.m;
  if (GRAD) {
    // reduce the gradient partials over the row slots of the warp
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
#pragma unroll
      for (int o = T; o < 32; o <<= 1) {
        g1[s] += __shfl_xor_sync(0xffffffffu, g1[s], o);
        g2[s] += __shfl_xor_sync(0xffffffffu, g2[s], o);
      }
    }
    if (W.rs == 0) {
#pragma unroll
      for (int s = 0; s < CPL; ++s) {
        sm.G1[W.gl * CPL + s] = g1[s];
        sm.G2[W.gl * CPL + s] = g2[s];
      }
    }
  }
  __syncwarp();
  // delta'(B + C delta / 2) and, with GRAD, the per-column gradient
  const int p = a.p;
  double qlin = 0.0;
  const CT ta = (CT)temp, ta2 = (CT)(temp * temp * nm * nm), tnm = (CT)(temp * nm);
  const CT cdbar = (CT)dbar;
  for (int c = W.lane; c < p; c += 32) {
    CT cd = CT(0);
    for (int k = 0; k < p; ++k) cd = fma(ldg_ct<CT>(a.C_ct, k * p + c), sm.dl[k], cd);
    const CT bc = ldg_ct<CT>(a.B_ct, c), dc = sm.dl[c];
    qlin += (double)(dc * (bc + CT(0.5) * cd));
    if (GRAD) {
      const CT G1 = sm.G1[c], G2 = sm.G2[c];
      const CT pg = -(sm.th[c] - ldg_ct<CT>(a.mu_ct, c)) * ldg_ct<CT>(a.ivar_ct, c);
      sm.g[c] = ta * (bc + cd) + tnm * G1 - ta2 * (G2 - cdbar * G1) + pg;
    }
  }
  qlin = warp_sum(qlin);
  ell = a.A + qlin + nm * S;
  sig2 = nm * nm * (Q - S * S / (double)a.m);
  __syncwarp();
}

template <typename CT> __device__ __forceinline__ double log_prior_warp(const EstArgs &a,
                                                                         const CT *th) {
  double lp = 0.0;
  for (int c = threadIdx.x & 31; c < a.p; c += 32) {
    const double r = (double)th[c] - (double)ldg_ct<CT>(a.mu_ct, c);
    lp += -0.5 * r * r * (double)ldg_ct<CT>(a.ivar_ct, c);
  }
  return warp_sum(lp) + a.log_prior_const;
}

// sm.dl = theta - theta_bar, and the lane slots of the evaluator
template <typename XT, int T, int CPL, int U>
__device__ __forceinline__ void refresh_delta(WarpEval<XT, T, CPL, U> &W, const EstArgs &a,
                                              WarpSmem<typename Store<XT>::CT> &sm) {
  using CT = typename Store<XT>::CT;
  for (int c = W.lane; c < a.p; c += 32) sm.dl[c] = sm.th[c] - ldg_ct<CT>(a.tb_ct, c);
  __syncwarp();
  W.load_slots(sm.dl, a.p, W.dl);
}

// ------------------------------------------------------------------------------------------------
// Kernel 1: the plain estimator on caller particles (loglik_est / loglik_grad, cache refresh).
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_estimate(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;  // whole warp leaves together; no block-level barriers follow
  WarpEval<XT, T, CPL, U> W;
  const int slots = T * CPL;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U>::RING), a.p, slots);
  W.load_slots(reinterpret_cast<const CT *>(a.tb_ct), a.p, W.tb);
  const CT *th = reinterpret_cast<const CT *>(a.theta) + (int64_t)i * a.p;
  for (int c = W.lane; c < a.p; c += 32) sm.th[c] = th[c];
  __syncwarp();
  refresh_delta(W, a, sm);
  const double temp = a.a_from_state ? a.st->a : a.a_host;
  const int32_t *idx = a.u + (int64_t)i * a.m;
  double ell, sig2;
  double *blk = a.blk ? a.blk + (int64_t)i * a.G * 2 : nullptr;
  if (a.grad) {
    if (blk)
      eval_particle<XT, T, CPL, U, true, true>(W, a, idx, sm, temp, blk, ell, sig2);
    else
      eval_particle<XT, T, CPL, U, true, false>(W, a, idx, sm, temp, nullptr, ell, sig2);
    CT *g = reinterpret_cast<CT *>(a.grad) + (int64_t)i * a.p;
    for (int c = W.lane; c < a.p; c += 32) g[c] = sm.g[c];
  } else {
    if (blk)
      eval_particle<XT, T, CPL, U, false, true>(W, a, idx, sm, temp, blk, ell, sig2);
    else
      eval_particle<XT, T, CPL, U, false, false>(W, a, idx, sm, temp, nullptr, ell, sig2);
  }
  if (W.lane == 0) {
    if (a.ell) a.ell[i] = ell;
    if (a.sig2) a.sig2[i] = sig2;
    if (!isfinite(ell) || !isfinite(sig2)) set_err(a.st, kErrNonFinite);
  }
}

// ------------------------------------------------------------------------------------------------
// Kernel 2: block pseudo-marginal update of u (Algorithm 1 step 1, Eq. acc_prop_u).
// One block g ~ U{0..G-1} of the floor partition is redrawn iid from p(u); only its m/G rows are
// gathered (at the current theta). The other blocks' sums come from the cache, and because the
// control-variate total sum_k q_k(theta) is common to both estimates it cancels in the ratio:
//   log r = a (n/m)(S_g* - S_g) - (a^2/2)(sigma2* - sigma2).
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_upm(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  WarpEval<XT, T, CPL, U> W;
  const int slots = T * CPL;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U>::RING), a.p, slots);
  const uint32_t smv = stage_move(a.stage, a.move);
  const Stream sblk(a.seed, kUpmBlock, smv, (uint32_t)i);
  const Stream sidx(a.seed, kUpmIdx, smv, (uint32_t)i);
  const int g = (int)draw_index(sblk.draw(0), (uint64_t)a.G);
  const int j0 = (int)(((int64_t)g * a.m) / a.G), j1 = (int)(((int64_t)(g + 1) * a.m) / a.G);
  const int nb = j1 - j0;
  int32_t *unew = a.unew + (int64_t)i * a.maxblk;
  for (int t = 2 * W.lane; t < nb; t += 64) {
    uint64_t r0, r1;
    sidx.pair((uint32_t)(t >> 1), r0, r1);
    unew[t] = (int32_t)draw_index(r0, (uint64_t)a.n);
    if (t + 1 < nb) unew[t + 1] = (int32_t)draw_index(r1, (uint64_t)a.n);
  }
  W.load_slots(reinterpret_cast<const CT *>(a.tb_ct), a.p, W.tb);
  const CT *th = reinterpret_cast<const CT *>(a.theta) + (int64_t)i * a.p;
  for (int c = W.lane; c < a.p; c += 32) sm.th[c] = th[c];
  __syncwarp();
  refresh_delta(W, a, sm);
  CT sd = CT(0), sd2 = CT(0);
  W.template rows<false>(reinterpret_cast<const XT *>(a.Xp), a.S, a.Yo, a.p, a.n, unew, 0, nb,
                         a.fam,
                         (CT)a.inv_s2, nullptr, nullptr, sd, sd2, a.st);
  const double Sg = warp_sum((double)sd), Qg = warp_sum((double)sd2);
  double *blk = a.blk + (int64_t)i * a.G * 2;
  // totals over blocks from the cache (lanes over blocks)
  double St = 0.0, Qt = 0.0;
  for (int h = W.lane; h < a.G; h += 32) {
    St += blk[2 * h];
    Qt += blk[2 * h + 1];
  }
  St = warp_sum(St);
  Qt = warp_sum(Qt);
  const double Sold = blk[2 * g], Qold = blk[2 * g + 1];
  const double temp = a.st->a;
  const double nm = (double)a.n / (double)a.m;
  const double Sn = St - Sold + Sg, Qn = Qt - Qold + Qg;
  const double ell0 = a.ell[i], sig0 = a.sig2[i];
  const double ell1 = ell0 + nm * (Sg - Sold);
  const double sig1 = nm * nm * (Qn - Sn * Sn / (double)a.m);
  const double log_r = temp * (ell1 - ell0) - 0.5 * temp * temp * (sig1 - sig0);
  const Stream smh(a.seed, kMhU, smv, (uint32_t)i);
  const double Uu = draw_uniform(smh.draw(0));
  const bool acc = log(Uu) < log_r;
  if (acc) {
    int32_t *ui = a.u_mut + (int64_t)i * a.m + j0;
    for (int t = W.lane; t < nb; t += 32) ui[t] = unew[t];
    if (W.lane == 0) {
      a.ell[i] = ell1;
      a.sig2[i] = sig1;
      blk[2 * g] = Sg;
      blk[2 * g + 1] = Qg;
      atomicAdd(&a.st->acc_u, 1ull);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Kernel 3: one HMC move of theta given u (Algorithm 1 step 2), the whole trajectory in one launch.
// rho = L^{-T} z (so rho ~ N(0, Sigma^{-1}) = N(0, H)), L leapfrog steps
//   rho += eps/2 g;  theta += eps Sigma rho;  g = grad(theta);  rho += eps/2 g
// then accept with probability min(1, exp(H0 - H1)), H = -log target + rho'Sigma rho / 2 (FP64).
// On acceptance theta, l_hat, sigma2_hat and the block sums at the end point replace the cache.
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_hmc(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  WarpEval<XT, T, CPL, U> W;
  const int slots = T * CPL;
  const int p = a.p;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U>::RING), p, slots);
  const uint32_t smv = stage_move(a.stage, a.move);
  const double temp = a.st->a;
  const CT eps = (CT)a.st->eps;
  W.load_slots(reinterpret_cast<const CT *>(a.tb_ct), p, W.tb);
  CT *th_g = reinterpret_cast<CT *>(a.theta_out) + (int64_t)i * p;
  for (int c = W.lane; c < p; c += 32) sm.th[c] = th_g[c];
  // momentum: z ~ N(0, I) in sm.v, rho = Linv' z  (rho_r = sum_c Linv[c, r] z_c, c >= r)
  const Stream smom(a.seed, kMomentum, smv, (uint32_t)i);
  for (int c = W.lane; c < p; c += 32) sm.v[c] = (CT)stream_normal(smom, (uint32_t)c);
  __syncwarp();
  for (int r = W.lane; r < p; r += 32) {
    CT acc = CT(0);
    for (int c = r; c < p; ++c) acc = fma(ldg_ct<CT>(a.Linv_ct, c * p + r), sm.v[c], acc);
    sm.rho[r] = acc;
  }
  __syncwarp();
  auto kinetic = [&]() -> double {  // rho' Sigma rho / 2
    double k = 0.0;
    for (int r = W.lane; r < p; r += 32) {
      CT acc = CT(0);
      for (int c = 0; c < p; ++c) acc = fma(ldg_ct<CT>(a.Sigma_ct, c * p + r), sm.rho[c], acc);
      k += (double)sm.rho[r] * (double)acc;
    }
    return 0.5 * warp_sum(k);
  };
  const double kin0 = kinetic();
  refresh_delta(W, a, sm);
  const int32_t *idx = a.u + (int64_t)i * a.m;
  double ell0, sig0;
  eval_particle<XT, T, CPL, U, true, false>(W, a, idx, sm, temp, nullptr, ell0, sig0);
  const double H0 = -(temp * ell0 - 0.5 * temp * temp * sig0 + log_prior_warp<CT>(a, sm.th)) + kin0;
  double ell1 = ell0, sig1 = sig0;
  double *bprop = a.blk_prop + (int64_t)i * a.G * 2;
  for (int l = 0; l < a.L; ++l) {
    for (int c = W.lane; c < p; c += 32) sm.rho[c] += CT(0.5) * eps * sm.g[c];
    __syncwarp();
    for (int r = W.lane; r < p; r += 32) {
      CT acc = CT(0);
      for (int c = 0; c < p; ++c) acc = fma(ldg_ct<CT>(a.Sigma_ct, c * p + r), sm.rho[c], acc);
      sm.v[r] = acc;
    }
    __syncwarp();
    for (int c = W.lane; c < p; c += 32) sm.th[c] += eps * sm.v[c];
    __syncwarp();
    refresh_delta(W, a, sm);
    if (l == a.L - 1)
      eval_particle<XT, T, CPL, U, true, true>(W, a, idx, sm, temp, bprop, ell1, sig1);
    else
      eval_particle<XT, T, CPL, U, true, false>(W, a, idx, sm, temp, nullptr, ell1, sig1);
    for (int c = W.lane; c < p; c += 32) sm.rho[c] += CT(0.5) * eps * sm.g[c];
    __syncwarp();
  }
  const double H1 =
      -(temp * ell1 - 0.5 * temp * temp * sig1 + log_prior_warp<CT>(a, sm.th)) + kinetic();
  const Stream smh(a.seed, kMhTheta, smv, (uint32_t)i);
  const double Uu = draw_uniform(smh.draw(0));
  const bool acc = log(Uu) < H0 - H1;  // false when H1 is NaN: the move is rejected
  if (acc) {
    for (int c = W.lane; c < p; c += 32) th_g[c] = sm.th[c];
    double *blk = a.blk + (int64_t)i * a.G * 2;
    for (int h = W.lane; h < 2 * a.G; h += 32) blk[h] = bprop[h];
    if (W.lane == 0) {
      a.ell[i] = ell1;
      a.sig2[i] = sig1;
      atomicAdd(&a.st->acc_theta, 1ull);
    }
  }
}

// ------------------------------------------------------------------------------------------------
// Launch helpers
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS>
inline int launch_tile(int op, const EstArgs &a, cudaStream_t s) {
  using CT = typename Store<XT>::CT;
  const size_t smem = (size_t)WARPS * warp_smem_bytes<XT, T, CPL, U>(a.p);
  const dim3 grid((a.B + WARPS - 1) / WARPS), block(WARPS * 32);
  if (a.B <= 0) return 0;
  cudaError_t e;
  if (op == 0) {
    e = cudaFuncSetAttribute(k_estimate<XT, T, CPL, U, WARPS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_estimate<XT, T, CPL, U, WARPS><<<grid, block, smem, s>>>(a);
  } else if (op == 1) {
    e = cudaFuncSetAttribute(k_upm<XT, T, CPL, U, WARPS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_upm<XT, T, CPL, U, WARPS><<<grid, block, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_hmc<XT, T, CPL, U, WARPS>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_hmc<XT, T, CPL, U, WARPS><<<grid, block, smem, s>>>(a);
  }
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

}  // namespace subsmc
