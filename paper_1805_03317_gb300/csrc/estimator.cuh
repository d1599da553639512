// Warp-per-particle subsampled estimator and the kernels built on it.
//
// One warp owns one particle. Its m subsampled rows are gathered straight from the packed row
// copy of the data (WarpEval below: 32 rows per sweep, one row owned per lane, covariates split
// over groups of T lanes). Per row the warp forms D = x'(theta - theta_bar), evaluates the
// increment-form terms d and r (device.cuh) from the row's stored constants at the centre, and
// accumulates, with e = d - K for a warp-uniform shift K (the d of the particle's first row),
//   sum e, sum e^2                 (per block of u when the block cache is refreshed)
//   sum r x, sum e r x             (gradient partials, kept in registers)
// which give (Sec. 3.2, Eq. difference_estimator_logl)
//   l_hat      = A + B'delta + delta'C delta/2 + (n/m)(sum e + m K)
//   sigma2_hat = (n^2/m^2) (sum e^2 - (sum e)^2/m)            (clamped at 0)
//   grad       = a (B + C delta + (n/m) sum r x) - a^2 (n^2/m^2)(sum e r x - ebar sum r x) - (theta-mu)/v
// The last line is the exact gradient of a*l_hat - a^2/2*sigma2_hat + log p(theta) for fixed u.
// The shift makes the one-pass variance stable (shifted data, Chan, Golub & LeVeque 1983): far
// from the centre the d_j share a large mean, and sum d^2 - (sum d)^2/m taken directly would
// cancel in FP32; sum e^2 - (sum e)^2/m only loses (ebar/sd(d))^2, and ebar is O(sd(d)). Block
// sums of the cache keep the exact FP64 (sum d, sum d^2) form, rebuilt from the shifted FP32
// sums per block: sum d = sum e + n_g K, sum d^2 = sum e^2 + 2 K sum e + n_g K^2.
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

// Per-row traffic of the forward/backward pair behind the autograd binding. MODE 1 (forward):
// d_j and r_j of every row are written to dsave/rsave [m]. MODE 2 (backward): no x'delta and no
// family terms; row j's weight is r_j (c1 + c2 (d_j - dbar)) from the saved values, and the
// gradient partials accumulate weight * x (g1 only).
template <typename CT> struct RowIO {
  CT *dsave = nullptr, *rsave = nullptr;
  const CT *dsaved = nullptr, *rsaved = nullptr;
  CT c1 = CT(0), c2 = CT(0), dbar = CT(0);
};

// Streamed rows. A warp takes its particle's rows 32 at a time (a sweep) and lane l owns row l of
// the sweep. For the covariates the warp splits into 32/T groups of T lanes: group r covers rows
// rT .. rT+T-1 of the sweep, and lane g of the group holds element slots g*CPL .. g*CPL+CPL-1 of
// each of them. Per sweep a lane forms partial x'delta over its slots for its group's T rows; a
// reduce-scatter inside the group leaves every lane the full D of the row it owns; the lane
// evaluates d and r for that row alone, from the constants in the row's tail; an all-gather inside
// the group then hands every lane r and d*r of the group's rows for the gradient partials over its
// slots. So the family terms are evaluated once per row, not once per lane of the row.
//
// Rows reach the lanes through a per-warp ring of NST sweeps in shared memory, filled by 16-byte
// cp.async copies issued NST-1 sweeps ahead (the row indices one sweep further ahead still). The
// lanes of a group copy a row's vectors contiguously (coalesced): covariate chunks into their own
// ring slots, the tail vector into the tail slot of the row's owner, which reads it after a warp
// barrier. (When the tiles' chunks end before the tail, the owner copies its tail itself.)
// Chunk vectors are XOR-swizzled so that 128-bit reads of 8 consecutive lanes hit distinct bank
// groups; chunk vectors that lie past the covariates are never copied and stay zero.
template <typename XT, int T, int CPL, int NST, bool PIPE = false>
struct WarpEval {
  using SD = Store<XT>;
  using CT = typename SD::CT;
  static constexpr int NV = CPL / SD::VEC;               // 16-byte vectors per lane per row
  static constexpr int TB = (int)sizeof(RowC<CT>);       // tail bytes per row
  static constexpr int XBYTES = 32 * T * NV * 16;        // covariate chunks of one sweep
  static constexpr int STAGE = XBYTES + 32 * TB;         // one sweep: chunks, then owned tails
  static constexpr int RING = NST * STAGE;               // ring bytes per warp
  static_assert(CPL % SD::VEC == 0, "CPL must be a whole number of 16-byte vectors");
  static_assert(NV == 1 || NV == 2 || NV == 3 || NV == 4 || NV == 8, "vectors per lane");
  static_assert(T >= 1 && T <= 32 && (T & (T - 1)) == 0, "T must be a power of two");
  static_assert(NST >= 2 && NST <= 32, "ring depth");

  CT dl[CPL];
  int lane, gl, gb, swz, tail_off;
  unsigned cmask;        // bit v: chunk vector v of this lane holds covariates (is copied)
  unsigned tmask;        // bit v: chunk vector v of this lane is a tail vector (copied to the tail slot)
  bool tail_in_chunks;   // the tail vectors fall inside the group's chunks (else owners copy them)
  unsigned char *ring;

  // ring: this warp's RING bytes (16-byte aligned). Yo: element at which the row's tail starts.
  __device__ __forceinline__ void init(unsigned char *ring_, int Yo) {
    lane = threadIdx.x & 31;
    gl = lane & (T - 1);
    gb = lane & ~(T - 1);
    swz = (NV == 2 || NV == 4 || NV == 8) ? ((lane / (8 / NV)) & (NV - 1)) : 0;
    ring = ring_;
    tail_off = Yo * (int)sizeof(XT);
    const int nvx = tail_off / 16;
    tail_in_chunks = nvx + TB / 16 <= T * NV;
    cmask = tmask = 0u;
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      const int vi = gl * NV + v;
      if (vi < nvx) cmask |= 1u << v;
      else if (tail_in_chunks && vi < nvx + TB / 16) tmask |= 1u << v;
    }
    for (int st = 0; st < NST; ++st)
#pragma unroll
      for (int t = 0; t < T; ++t)
#pragma unroll
        for (int v = 0; v < NV; ++v)
          if (!((cmask >> v) & 1u))
            *reinterpret_cast<uint4 *>(chunk(st, t, v)) = make_uint4(0u, 0u, 0u, 0u);
  }
  __device__ __forceinline__ unsigned char *chunk(int st, int t, int v) const {
    return ring + st * STAGE + ((t * 32 + lane) * NV + (v ^ swz)) * 16;
  }
  __device__ __forceinline__ unsigned char *tail(int st, int q) const {
    return ring + st * STAGE + XBYTES + q * TB;
  }
  __device__ __forceinline__ unsigned char *tail(int st) const { return tail(st, lane); }
  // Slot s of this lane is element (column) gl*CPL + s of a packed row.
  __device__ __forceinline__ void load_slots(const CT *vec, int p, CT *dst) const {
#pragma unroll
    for (int s = 0; s < CPL; ++s) {
      const int c = gl * CPL + s;
      dst[s] = c < p ? vec[c] : CT(0);
    }
  }

  // One pass over rows idx[0..nrows). GRAD: accumulates the gradient partials sum r x, sum d r x
  // over this lane's slots into g1, g2. Returns S = sum d and Q = sum d^2 on every lane; BLOCKS
  // also writes per-block (sum d, sum d^2) of the floor partition of the nrows rows into G blocks
  // to blk_out[2G].
  // The sums are of e = d - K (returned in Ksh, warp-uniform: the d of row 0), so
  // Ssum = sum e and Qsum = sum e^2; g2 accumulates e r x. BLOCKS writes the unshifted FP64 block
  // sums (sum d, sum d^2) rebuilt from the shifted ones.
  template <bool GRAD, bool BLOCKS, int MODE = 0>
  __device__ __forceinline__ void rows(const XT *__restrict__ Xp, int S, int64_t n,
                                       const int32_t *idx, int nrows, int fam, CT inv_s2, CT *g1,
                                       CT *g2, double *blk_out, int G, double &Ssum, double &Qsum,
                                       double &Ksh, DevState *st,
                                       const RowIO<CT> &io = RowIO<CT>(), int cv1 = 0) const {
    const int nsw = (nrows + 31) >> 5;
    // rows past the end copy the last row again (already on chip) and are masked out
    const int klast = nrows > 0 ? idx[nrows - 1] : 0;
    unsigned bad = 0u;  // bit b: the row this lane owns in ring stage b had an invalid index
    int kq = 0;         // index of this lane's row in the next sweep to issue
    auto fetch = [&](int s) {
      if (s < nsw) {
        const int j = (s << 5) + lane;
        kq = j < nrows ? idx[j] : klast;  // plain load: u-update indices are written by this warp
      }
    };
    auto issue = [&](int s) {
      if (s < nsw) {
        const int b = s % NST;
        int k = kq;
        if (k < 0 || (int64_t)k >= n) {
          if ((s << 5) + lane < nrows) set_err(st, kErrIndex);
          bad |= 1u << b;
          k = 0;
        } else {
          bad &= ~(1u << b);
        }
        if (!tail_in_chunks) {  // the owner fetches its row's tail itself (uncoalesced)
          const unsigned char *row = reinterpret_cast<const unsigned char *>(Xp + (int64_t)k * S);
#pragma unroll
          for (int q = 0; q < TB / 16; ++q) cp_async16(tail(b) + 16 * q, row + tail_off + 16 * q);
        }
#pragma unroll
        for (int t = 0; t < T; ++t) {
          const int kt = __shfl_sync(0xffffffffu, k, gb + t);
          const unsigned char *src =
              reinterpret_cast<const unsigned char *>(Xp + (int64_t)kt * S) + gl * (NV * 16);
          // the group's lanes read the row's vectors contiguously: covariate chunks go to this
          // lane's ring slots, tail vectors to the tail slot of the row's owner
#pragma unroll
          for (int v = 0; v < NV; ++v) {
            if (((cmask | tmask) >> v) & 1u) {  // one copy instruction for the whole group
              unsigned char *dst = ((cmask >> v) & 1u)
                                       ? chunk(b, t, v)
                                       : tail(b, gb + t) + (gl * NV + v) * 16 - tail_off;
              cp_async16(dst, src + 16 * v);
            }
          }
        }
      }
      cp_async_commit();  // one group per sweep (empty past the end) keeps the counting uniform
    };
    if (BLOCKS) {
      for (int h = lane; h < 2 * G; h += 32) blk_out[h] = 0.0;  // blocks with no rows stay zero
      __syncwarp();
    }
    CT sd = CT(0), sd2 = CT(0);
    double cs = 0.0, cq = 0.0;  // BLOCKS: shifted sums of the open block cg
    int cg = -1;
    CT K = CT(0);               // shift of the sums: d of row 0 (set at sweep 0)
    Ssum = Qsum = 0.0;
    // close block g: its unshifted FP64 sums from the shifted ones
    auto close_block = [&](int g) {
      const double ng = (double)((int)(((int64_t)(g + 1) * nrows) / G) -
                                 (int)(((int64_t)g * nrows) / G));
      const double k = (double)K;
      blk_out[2 * g] = fma(ng, k, cs);
      blk_out[2 * g + 1] = cq + k * fma(ng, k, 2.0 * cs);
    };
    // partial x'delta of the group's T rows over this lane's slots, reduce-scattered: the full D of
    // the row this lane owns
    auto phase1 = [&](int b) -> CT {
      CT pd[T];
#pragma unroll
      for (int t = 0; t < T; ++t) {
        CT x[CPL];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          SD::unpack(*reinterpret_cast<const uint4 *>(chunk(b, t, v)), &x[v * SD::VEC]);
        pd[t] = dot_slots<CPL>(x, dl);
      }
      int base = 0;
      reduce_scatter<T, T / 2, CT>(pd, lane, base);
      return pd[0];
    };
    // d and r of the owned row of sweep s (stage b) at D, masked past the end; sums of d, d^2
    auto terms = [&](int s, int b, CT D, CT &d, CT &r) {
      const int j = (s << 5) + lane;
      if constexpr (MODE == 2) {  // weight of the row from the saved forward values
        (void)D;
        d = CT(0);
        r = CT(0);
        if (j < nrows && !((bad >> b) & 1u))
          r = io.rsaved[j] * (io.c1 + io.c2 * (io.dsaved[j] - io.dbar));
        return;
      }
      const RowC<CT> c = *reinterpret_cast<const RowC<CT> *>(tail(b));
      // every lane evaluates a row here, so a warp vote is safe
      const bool short4 = __all_sync(0xffffffffu, fabs(D) <= CT(0.05));
      switch (fam) {
        case 0: row_incr<0, CT>(c, D, inv_s2, d, r, short4); break;
        case 1: row_incr<1, CT>(c, D, inv_s2, d, r); break;
        case 2: row_incr<2, CT>(c, D, inv_s2, d, r); break;
        case 3: row_incr<3, CT>(c, D, inv_s2, d, r); break;
        default: row_incr<4, CT>(c, D, inv_s2, d, r); break;
      }
      if (cv1) to_first_order(row_l2_any(fam, c, inv_s2), D, d, r);
      const bool valid = j < nrows && !((bad >> b) & 1u);
      if (!valid) {
        d = CT(0);
        r = CT(0);
      }
      if constexpr (MODE == 1) {
        if (j < nrows) {
          io.dsave[j] = d;
          io.rsave[j] = r;
        }
      }
      if (s == 0) K = __shfl_sync(0xffffffffu, d, 0);  // every lane is here at sweep 0
      d = valid ? d - K : CT(0);  // from here on d holds e = d - K
      if (BLOCKS) {  // block of row j: largest g with floor(g nrows / G) <= j
        const int r1 = min((s << 5) + 31, nrows - 1);
        const int gA = (int)(((unsigned)((s << 5) + 1) * (unsigned)G - 1u) / (unsigned)nrows);
        const int gB = (int)(((unsigned)(r1 + 1) * (unsigned)G - 1u) / (unsigned)nrows);
        const int gj =
            j < nrows ? (int)(((unsigned)(j + 1) * (unsigned)G - 1u) / (unsigned)nrows) : -1;
        for (int g = gA; g <= gB; ++g) {
          const CT bs = warp_sum(gj == g ? d : CT(0));
          const CT bq = warp_sum(gj == g ? d * d : CT(0));
          if (g != cg) {
            if (cg >= 0 && lane == 0) close_block(cg);
            cg = g;
            cs = cq = 0.0;
          }
          cs += (double)bs;
          cq += (double)bq;
          Ssum += (double)bs;
          Qsum += (double)bq;
        }
      } else {
        sd += d;
        sd2 = fma(d, d, sd2);
      }
    };
    // gradient partials over this lane's slots: all-gather r, d r of the group's rows
    auto phase2 = [&](int b, CT r, CT dr) {
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const CT rt = __shfl_sync(0xffffffffu, r, gb + t);
        const CT drt = __shfl_sync(0xffffffffu, dr, gb + t);
        CT x[CPL];
#pragma unroll
        for (int v = 0; v < NV; ++v)
          SD::unpack(*reinterpret_cast<const uint4 *>(chunk(b, t, v)), &x[v * SD::VEC]);
        axpy_slots<CPL>(rt, x, g1);
        if constexpr (MODE != 2) axpy_slots<CPL>(drt, x, g2);
      }
    };
    fetch(0);
#pragma unroll
    for (int q = 0; q < NST - 1; ++q) {
      issue(q);
      fetch(q + 1);
    }
    if constexpr (PIPE) {
      // Software pipelined: iteration s evaluates the terms of sweep s, then runs the partial
      // x'delta of sweep s+1 and the gradient partials of sweep s side by side (independent
      // instruction streams for the scheduler). Needs NST >= 3: stages of s and s+1 are read while
      // s+NST-1 is in flight.
      static_assert(!PIPE || NST >= 3, "pipelined sweeps need three ring stages");
      CT Dc = CT(0);
      if (nsw > 0) {
        cp_async_wait<NST - 2>();  // sweep 0 has landed
        if (tail_in_chunks) __syncwarp();  // tails were copied by other lanes of the group
        if (MODE != 2) Dc = phase1(0);
      }
      for (int s = 0; s < nsw; ++s) {
        const int b = s % NST;
        issue(s + NST - 1);
        fetch(s + NST);
        CT d, r;
        terms(s, b, Dc, d, r);
        cp_async_wait<NST - 2>();  // sweep s+1 has landed
        if (tail_in_chunks) __syncwarp();
        CT Dn = CT(0);
        if (MODE != 2 && s + 1 < nsw) Dn = phase1((s + 1) % NST);
        if (GRAD) phase2(b, r, d * r);
        Dc = Dn;
      }
    } else {
      for (int s = 0; s < nsw; ++s) {
        issue(s + NST - 1);
        fetch(s + NST);
        cp_async_wait<NST - 1>();  // this lane's copies of sweep s have landed
        if (tail_in_chunks) __syncwarp();  // tails were copied by other lanes of the group
        const int b = s % NST;
        const CT D = MODE == 2 ? CT(0) : phase1(b);
        CT d, r;
        terms(s, b, D, d, r);
        if (GRAD) {
          // the chunks are read again rather than held across the family terms (that would
          // cost T*CPL registers)
          asm volatile("" ::: "memory");
          phase2(b, r, d * r);
        }
      }
    }
    cp_async_wait<0>();
    if (BLOCKS) {
      if (cg >= 0 && lane == 0) close_block(cg);
    } else {
      Ssum = warp_sum((double)sd);
      Qsum = warp_sum((double)sd2);
    }
    Ksh = (double)K;
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
template <typename XT, int T, int CPL, int U, bool K, bool GRAD, bool BLOCKS, int MODE = 0>
__device__ __forceinline__ void eval_particle(const WarpEval<XT, T, CPL, U, K> &W, const EstArgs &a,
                                              const int32_t *idx, WarpSmem<typename Store<XT>::CT> &sm,
                                              double temp, double *blk_out, double &ell,
                                              double &sig2,
                                              const RowIO<typename Store<XT>::CT> &io =
                                                  RowIO<typename Store<XT>::CT>()) {
  using CT = typename Store<XT>::CT;
  const XT *Xp = reinterpret_cast<const XT *>(a.Xp);
  const CT inv_s2 = (CT)a.inv_s2;
  CT g1[CPL], g2[CPL];
#pragma unroll
  for (int s = 0; s < CPL; ++s) g1[s] = g2[s] = CT(0);
  double S, Q, Ks;  // sums of e = d - Ks and e^2, and the shift Ks
  W.template rows<GRAD, BLOCKS, MODE>(Xp, a.S, a.n, idx, a.m, a.fam, inv_s2, g1, g2, blk_out, a.G,
                                      S, Q, Ks, a.st, io, a.cv_order == 1);
  const double nm = (double)a.n / (double)a.m;
  const double dbar = S / (double)a.m;  // mean of e (the gradient partials hold e r x)
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
    if (W.gb == 0) {
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
  ell = (a.A_dev ? __ldg(a.A_dev) : a.A) + qlin + nm * fma((double)a.m, Ks, S);
  sig2 = nm * nm * fmax(0.0, Q - S * S / (double)a.m);
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
template <typename XT, int T, int CPL, int U, bool K>
__device__ __forceinline__ void refresh_delta(WarpEval<XT, T, CPL, U, K> &W, const EstArgs &a,
                                              WarpSmem<typename Store<XT>::CT> &sm) {
  using CT = typename Store<XT>::CT;
  for (int c = W.lane; c < a.p; c += 32) sm.dl[c] = sm.th[c] - ldg_ct<CT>(a.tb_ct, c);
  __syncwarp();
  W.load_slots(sm.dl, a.p, W.dl);
}

// Problem of global particle g: the last q with offsets[q] <= g (offsets ascending, offsets[0] = 0).
__device__ __forceinline__ int batch_problem(const int *offsets, int nprob, int g) {
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(offsets + mid) <= g)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

// ------------------------------------------------------------------------------------------------
// Kernel 1: the plain estimator on caller particles (loglik_est / loglik_grad, cache refresh).
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_estimate(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;  // whole warp leaves together; no block-level barriers follow
  WarpEval<XT, T, CPL, U, K> W;
  const int slots = T * CPL;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U, K>::RING), a.p, slots);
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
      eval_particle<XT, T, CPL, U, K, true, true>(W, a, idx, sm, temp, blk, ell, sig2);
    else
      eval_particle<XT, T, CPL, U, K, true, false>(W, a, idx, sm, temp, nullptr, ell, sig2);
    CT *g = reinterpret_cast<CT *>(a.grad) + (int64_t)i * a.p;
    for (int c = W.lane; c < a.p; c += 32) g[c] = sm.g[c];
  } else {
    if (blk)
      eval_particle<XT, T, CPL, U, K, false, true>(W, a, idx, sm, temp, blk, ell, sig2);
    else
      eval_particle<XT, T, CPL, U, K, false, false>(W, a, idx, sm, temp, nullptr, ell, sig2);
  }
  if (W.lane == 0) {
    if (a.ell) a.ell[i] = ell;
    if (a.sig2) a.sig2[i] = sig2;
    if (!isfinite(ell) || !isfinite(sig2)) set_err(a.st, kErrNonFinite);
  }
}

// ------------------------------------------------------------------------------------------------
// Forward/backward pair behind the autograd binding (Sec. 3.2 estimator, its exact gradient for
// fixed u). Forward: l_hat and sigma2_hat as loglik_est, and per row d_j, r_j saved to
// dsave/rsave [B, m]. Backward, for upstream gradients (g_l, g_s) of (l_hat, sigma2_hat):
//   dL/dtheta = g_l (B + C delta) + sum_j r_j [g_l n/m + g_s 2 (n/m)^2 (d_j - dbar)] x_j
// from the saved values and the rows gathered again by u (no family terms are re-evaluated).
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_fwdsave(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  WarpEval<XT, T, CPL, U, K> W;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U, K>::RING), a.p, T * CPL);
  const CT *th = reinterpret_cast<const CT *>(a.theta) + (int64_t)i * a.p;
  for (int c = W.lane; c < a.p; c += 32) sm.th[c] = th[c];
  __syncwarp();
  refresh_delta(W, a, sm);
  RowIO<CT> io;
  io.dsave = reinterpret_cast<CT *>(a.dsave) + (int64_t)i * a.m;
  io.rsave = reinterpret_cast<CT *>(a.rsave) + (int64_t)i * a.m;
  double ell, sig2;
  eval_particle<XT, T, CPL, U, K, false, false, 1>(W, a, a.u + (int64_t)i * a.m, sm, 1.0, nullptr,
                                                    ell, sig2, io);
  if (W.lane == 0) {
    a.ell[i] = ell;
    a.sig2[i] = sig2;
    if (!isfinite(ell) || !isfinite(sig2)) set_err(a.st, kErrNonFinite);
  }
}

template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_backward(EstArgs a) {
  using CT = typename Store<XT>::CT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  WarpEval<XT, T, CPL, U, K> W;
  const int p = a.p, m = a.m;
  unsigned char *wbase = smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(p);
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U, K>::RING), p, T * CPL);
  const CT *th = reinterpret_cast<const CT *>(a.theta) + (int64_t)i * p;
  for (int c = W.lane; c < p; c += 32) sm.th[c] = th[c];
  __syncwarp();
  refresh_delta(W, a, sm);
  RowIO<CT> io;
  io.dsaved = reinterpret_cast<const CT *>(a.dsave) + (int64_t)i * m;
  io.rsaved = reinterpret_cast<const CT *>(a.rsave) + (int64_t)i * m;
  double sd = 0.0;
  for (int j = W.lane; j < m; j += 32) sd += (double)io.dsaved[j];
  sd = warp_sum(sd);
  const double nm = (double)a.n / (double)m, gl = a.g_ell[i], gs = a.g_sig2[i];
  io.c1 = (CT)(gl * nm);
  io.c2 = (CT)(gs * 2.0 * nm * nm);
  io.dbar = (CT)(sd / (double)m);
  CT g1[CPL], g2[CPL];
#pragma unroll
  for (int e = 0; e < CPL; ++e) g1[e] = g2[e] = CT(0);
  double S_, Q_, K_;
  W.template rows<true, false, 2>(reinterpret_cast<const XT *>(a.Xp), a.S, a.n,
                                  a.u + (int64_t)i * m, m, a.fam, (CT)a.inv_s2, g1, g2, nullptr,
                                  a.G, S_, Q_, K_, a.st, io);
#pragma unroll
  for (int e = 0; e < CPL; ++e) {
#pragma unroll
    for (int o = T; o < 32; o <<= 1) g1[e] += __shfl_xor_sync(0xffffffffu, g1[e], o);
  }
  if (W.gb == 0) {
#pragma unroll
    for (int e = 0; e < CPL; ++e) sm.G1[W.gl * CPL + e] = g1[e];
  }
  __syncwarp();
  CT *gout = reinterpret_cast<CT *>(a.grad) + (int64_t)i * p;
  const CT cgl = (CT)gl;
  for (int c = W.lane; c < p; c += 32) {
    CT cd = CT(0);
    for (int k = 0; k < p; ++k) cd = fma(ldg_ct<CT>(a.C_ct, k * p + c), sm.dl[k], cd);
    gout[c] = cgl * (ldg_ct<CT>(a.B_ct, c) + cd) + sm.G1[c];
  }
}

// ------------------------------------------------------------------------------------------------
// Kernel 2: block pseudo-marginal update of u (Algorithm 1 step 1, Eq. acc_prop_u).
// One block g ~ U{0..G-1} of the floor partition is redrawn iid from p(u); only its m/G rows are
// gathered (at the current theta). The other blocks' sums come from the cache, and because the
// control-variate total sum_k q_k(theta) is common to both estimates it cancels in the ratio:
//   log r = a (n/m)(S_g* - S_g) - (a^2/2)(sigma2* - sigma2).
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__device__ __forceinline__ void upm_body(const EstArgs &a, int i, unsigned char *wbase) {
  using CT = typename Store<XT>::CT;
  WarpEval<XT, T, CPL, U, K> W;
  const int slots = T * CPL;
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U, K>::RING), a.p, slots);
  const uint32_t smv = stage_move(a.stage_dev ? a.st->stage : a.stage, a.move);
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
  const CT *th = reinterpret_cast<const CT *>(a.theta) + (int64_t)i * a.p;
  for (int c = W.lane; c < a.p; c += 32) sm.th[c] = th[c];
  __syncwarp();
  refresh_delta(W, a, sm);
  double Se, Qe, Ks;
  W.template rows<false, false>(reinterpret_cast<const XT *>(a.Xp), a.S, a.n, unew, nb, a.fam,
                                (CT)a.inv_s2, nullptr, nullptr, nullptr, 0, Se, Qe, Ks, a.st,
                                RowIO<CT>(), a.cv_order == 1);
  // the new block's FP64 (sum d, sum d^2) from the shifted sums of e = d - Ks
  const double Sg = fma((double)nb, Ks, Se), Qg = Qe + Ks * fma((double)nb, Ks, 2.0 * Se);
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
  const double sig1 = nm * nm * fmax(0.0, Qn - Sn * Sn / (double)a.m);
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
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_upm(EstArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  upm_body<XT, T, CPL, U, WARPS, K>(a, a.i0 + i,
                                  smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p));
}
// All particles of a batch of independent posteriors in one launch: the global warp index picks
// the problem (offsets: first particle of each problem) and the particle within it; per-warp
// shared memory has the batch's largest stride.
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_upm_batch(BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * WARPS + warp;
  if (g >= b.total) return;
  const int q = batch_problem(b.offsets, b.nprob, g);
  upm_body<XT, T, CPL, U, WARPS, K>(b.probs[q], g - b.offsets[q],
                                  smem_raw + (size_t)warp * b.wstride);
}

// ------------------------------------------------------------------------------------------------
// Kernel 3: one HMC move of theta given u (Algorithm 1 step 2), the whole trajectory in one launch.
// rho = L^{-T} z (so rho ~ N(0, Sigma^{-1}) = N(0, H)), L leapfrog steps
//   rho += eps/2 g;  theta += eps Sigma rho;  g = grad(theta);  rho += eps/2 g
// then accept with probability min(1, exp(H0 - H1)), H = -log target + rho'Sigma rho / 2 (FP64).
// On acceptance theta, l_hat, sigma2_hat and the block sums at the end point replace the cache.
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__device__ __forceinline__ void hmc_body(const EstArgs &a, int i, unsigned char *wbase) {
  using CT = typename Store<XT>::CT;
  WarpEval<XT, T, CPL, U, K> W;
  const int slots = T * CPL;
  const int p = a.p;
  W.init(wbase, a.Yo);
  WarpSmem<CT> sm(reinterpret_cast<CT *>(wbase + WarpEval<XT, T, CPL, U, K>::RING), p, slots);
  const uint32_t smv = stage_move(a.stage_dev ? a.st->stage : a.stage, a.move);
  const double temp = a.st->a;
  // random walk: the proposal scale itself; HMC: the particle's (jittered) step size
  const CT eps = a.rw ? (CT)a.st->eps
                      : (CT)jittered_eps(a.st->eps, a.eps_jitter, a.seed, smv, (uint32_t)i);
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
  const int32_t *idx = a.u + (int64_t)i * a.m;
  double *bprop = a.blk_prop + (int64_t)i * a.G * 2;
  if (a.rw) {  // random-walk Metropolis: theta* = theta + eps Sigma rho ~ N(theta, eps^2 Sigma)
    for (int r = W.lane; r < p; r += 32) {
      CT acc = CT(0);
      for (int c = 0; c < p; ++c) acc = fma(ldg_ct<CT>(a.Sigma_ct, c * p + r), sm.rho[c], acc);
      sm.v[r] = acc;
    }
    __syncwarp();
    for (int c = W.lane; c < p; c += 32) {  // sm.v keeps the proposal itself
      sm.v[c] = fma(eps, sm.v[c], sm.th[c]);
      sm.th[c] = sm.v[c];
    }
    __syncwarp();
    refresh_delta(W, a, sm);
    double ell1, sig1;
    eval_particle<XT, T, CPL, U, K, false, true>(W, a, idx, sm, temp, bprop, ell1, sig1);
    // the current state's estimates are the cache (same u); the momentum is not changed, so
    // the kinetic terms cancel and the MH ratio is the ratio of the targets
    const double lp1 = log_prior_warp<CT>(a, sm.th);
    __syncwarp();
    for (int c = W.lane; c < p; c += 32) sm.th[c] = th_g[c];
    __syncwarp();
    const double lp0 = log_prior_warp<CT>(a, sm.th);
    const double ell0 = a.ell[i], sig0 = a.sig2[i];
    const double t1 = temp * ell1 - 0.5 * temp * temp * sig1 + lp1;
    const double t0 = temp * ell0 - 0.5 * temp * temp * sig0 + lp0;
    const Stream smh(a.seed, kMhTheta, smv, (uint32_t)i);
    const double Uu = draw_uniform(smh.draw(0));
    if (log(Uu) < t1 - t0) {  // false when t1 is NaN: the move is rejected
      for (int c = W.lane; c < p; c += 32) th_g[c] = sm.v[c];
      double *blk = a.blk + (int64_t)i * a.G * 2;
      for (int h = W.lane; h < 2 * a.G; h += 32) blk[h] = bprop[h];
      if (W.lane == 0) {
        a.ell[i] = ell1;
        a.sig2[i] = sig1;
        atomicAdd(&a.st->acc_theta, 1ull);
      }
    }
    return;
  }
  const double kin0 = kinetic();
  refresh_delta(W, a, sm);
  double ell0, sig0;
  eval_particle<XT, T, CPL, U, K, true, false>(W, a, idx, sm, temp, nullptr, ell0, sig0);
  const double H0 = -(temp * ell0 - 0.5 * temp * temp * sig0 + log_prior_warp<CT>(a, sm.th)) + kin0;
  double ell1 = ell0, sig1 = sig0;
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
      eval_particle<XT, T, CPL, U, K, true, true>(W, a, idx, sm, temp, bprop, ell1, sig1);
    else
      eval_particle<XT, T, CPL, U, K, true, false>(W, a, idx, sm, temp, nullptr, ell1, sig1);
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
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_hmc(EstArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * WARPS + warp;
  if (i >= a.B) return;
  hmc_body<XT, T, CPL, U, WARPS, K>(a, a.i0 + i,
                                  smem_raw + (size_t)warp * warp_smem_bytes<XT, T, CPL, U>(a.p));
}
// All particles of a batch of independent posteriors in one launch: the global warp index picks
// the problem (offsets: first particle of each problem) and the particle within it; per-warp
// shared memory has the batch's largest stride.
template <typename XT, int T, int CPL, int U, int WARPS, bool K>
__global__ void __launch_bounds__(WARPS * 32) k_hmc_batch(BatchArgs b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int warp = threadIdx.x >> 5;
  const int g = blockIdx.x * WARPS + warp;
  if (g >= b.total) return;
  const int q = batch_problem(b.offsets, b.nprob, g);
  hmc_body<XT, T, CPL, U, WARPS, K>(b.probs[q], g - b.offsets[q],
                                  smem_raw + (size_t)warp * b.wstride);
}

// ------------------------------------------------------------------------------------------------
// Launch helpers
// ------------------------------------------------------------------------------------------------
template <typename XT, int T, int CPL, int U, int WARPS, bool K = false>
inline int launch_tile(int op, const EstArgs &a, cudaStream_t s) {
  using CT = typename Store<XT>::CT;
  const size_t smem = (size_t)WARPS * warp_smem_bytes<XT, T, CPL, U>(a.p);
  const dim3 grid((a.B + WARPS - 1) / WARPS), block(WARPS * 32);
  if (a.B <= 0) return 0;
  cudaError_t e;
  if (op == 0) {
    e = cudaFuncSetAttribute(k_estimate<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_estimate<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(a);
  } else if (op == 1) {
    e = cudaFuncSetAttribute(k_upm<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_upm<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(a);
  } else if (op == 2) {
    e = cudaFuncSetAttribute(k_hmc<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_hmc<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(a);
  } else if (op == 3) {
    e = cudaFuncSetAttribute(k_fwdsave<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_fwdsave<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(k_backward<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_backward<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(a);
  }
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

// Batched launch over all particles of a batch: op 1 = u-update, 2 = HMC move.
template <typename XT, int T, int CPL, int U, int WARPS, bool K = false>
inline int launch_tile_batch(int op, const BatchArgs &b, cudaStream_t s) {
  const size_t smem = (size_t)WARPS * b.wstride;
  const dim3 grid((b.total + WARPS - 1) / WARPS), block(WARPS * 32);
  if (b.total <= 0) return 0;
  cudaError_t e;
  if (op == 1) {
    e = cudaFuncSetAttribute(k_upm_batch<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_upm_batch<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(b);
  } else {
    e = cudaFuncSetAttribute(k_hmc_batch<XT, T, CPL, U, WARPS, K>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) k_hmc_batch<XT, T, CPL, U, WARPS, K><<<grid, block, smem, s>>>(b);
  }
  if (e != cudaSuccess) return (int)e;
  return (int)cudaGetLastError();
}

}  // namespace subsmc
