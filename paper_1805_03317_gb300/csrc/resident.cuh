// HMC trajectory with the particle's subsample resident in shared memory (Algorithm 1 step 2).
//
// u is fixed for the whole trajectory, so the m rows x_{u_j} are gathered once per particle
// (cp.async, 16-byte copies) and kept in shared memory, together with each row's stored
// control-variate constants (its tail: they depend on eta_bar_j and y_j only). The L + 1 estimator passes
// then read shared memory: one lane per row, D_j = x_j'(theta - theta_bar) and the increment terms
// d_j, r_j (device.cuh), gradient partials in registers, a shuffle reduce-scatter per warp and one
// CTA barrier per pass (partials double-buffered). Every warp then assembles the totals and the
// gradient and runs the leapfrog update itself, with theta, rho and the gradient held one column
// per lane (lane l also holds column l + 32 in tiles wider than 32 slots), so no warp waits for
// another between passes. One CTA handles one particle at a time and loops over particles
// (persistent grid).
//
// Sums over rows are of e_j = d_j - K with a CTA-uniform shift K near the subsample mean of d: the
// cached mean for the first pass, then the previous pass's mean (shifted data: Chan, Golub &
// LeVeque 1983). sigma2_hat = (n/m)^2 (sum e^2 - (sum e)^2/m) then stays accurate in FP32 partial
// sums where the d_j share a large mean (particles far from the centre), and the gradient's
// sum (d_j - dbar) r_j x_j is formed as sum e_j r_j x_j - ebar sum r_j x_j without that cancellation.
// The block cache keeps FP64 (sum d, sum d^2), rebuilt from the shifted block sums.
#pragma once

#include "estimator.cuh"

namespace subsmc {

// Shared-memory plan of one CTA.
struct ResPlan {
  int rb;    // bytes per resident row (covariates only): an odd multiple of 16 (conflict-free LDS.128)
  int nvec;  // 16-byte vectors of covariates per row (copied from the packed row)
  int nvl;   // 16-byte vectors the tile's CPL slots read (>= nvec; the extra ones are zero-filled)
  int off_consts, off_d, off_vec, off_red, off_redd, off_blk, off_mat, off_k, off_h, total;
};

// Constants of one launch of a problem (temperature, n/m, stage counter), computed once per
// problem by one thread instead of once per particle by every thread.
template <typename CT> struct alignas(16) ResK {
  double temp, nm, inv_m;
  CT ta, ta2, tnm;
  uint32_t smv;
};

inline __host__ __device__ int round16(int v) { return (v + 15) & ~15; }

template <typename CT>
inline ResPlan res_plan(int p, int m, int G, int esz, int warps, int cpl) {
  ResPlan P;
  const int xb = round16(p * esz), xl = round16(cpl * esz);
  P.nvec = xb / 16;
  P.nvl = xl / 16;
  P.rb = ((xl / 16) % 2 == 0) ? xl + 16 : xl;
  int off = m * P.rb;
  P.off_consts = off;
  off = round16(off + m * (int)sizeof(RowC<CT>));
  P.off_d = off;
  off = round16(off + m * (int)sizeof(CT));
  P.off_vec = off;  // initial momentum [cpl]
  off = round16(off + cpl * (int)sizeof(CT));
  P.off_red = off;  // two buffers of [warps][2 cpl] gradient partials
  off = round16(off + 2 * warps * 2 * cpl * (int)sizeof(CT));
  P.off_redd = off;  // two buffers of [warps][2] sums of d, d^2
  off = round16(off + 2 * warps * 2 * (int)sizeof(double));
  P.off_blk = off;
  off = round16(off + G * 2 * (int)sizeof(double));
  P.off_mat = off;  // C and Sigma, zero-padded to [cpl, cpl], state type
  off = round16(off + 2 * cpl * cpl * (int)sizeof(CT));
  P.off_k = off;
  off = round16(off + (int)sizeof(ResK<CT>));
  P.off_h = off;  // [3] log p(theta_0), log p(theta_L), log U of the MH test
  off = round16(off + 3 * (int)sizeof(double));
  P.total = off;
  return P;
}

__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// CPL covariate slots of a resident row; CPL need not be a multiple of the 16-byte vector width
// (the row holds whole vectors, zero-padded, and the unused tail of the last one is dropped).
template <typename XT, int CPL>
__device__ __forceinline__ void load_res_row(const unsigned char *row,
                                             typename Store<XT>::CT *x) {
  using SD = Store<XT>;
  using CT = typename SD::CT;
  constexpr int NV = CPL / SD::VEC, REM = CPL % SD::VEC;
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const uint4 w = *reinterpret_cast<const uint4 *>(row + 16 * v);
    SD::unpack(w, x + v * SD::VEC);
  }
  if constexpr (REM > 0) {
    CT t[SD::VEC];
    SD::unpack(*reinterpret_cast<const uint4 *>(row + 16 * NV), t);
#pragma unroll
    for (int e = 0; e < REM; ++e) x[NV * SD::VEC + e] = t[e];
  }
}

// One particle's trajectory: particle i of the problem described by a. reload: the CTA's previous
// particle belonged to another problem (or there was none), so the C and Sigma tiles are loaded.
// Lane l of every warp holds columns l, l + 32, .. of theta, rho and the gradient (NC per lane).
template <typename XT, int CPL, int WARPS>
__device__ __forceinline__ void res_particle(const EstArgs &a, int i, bool reload,
                                             const ResPlan &P) {
  using SD = Store<XT>;
  using CT = typename SD::CT;
  constexpr int NC = (CPL + 31) / 32;
  static_assert(NC <= 2, "at most two columns per lane");
  // the warps that take the log prior and the log of the MH uniform (warp 0: the kinetic energy)
  constexpr int kWarpP = WARPS > 1 ? 1 : 0, kWarpU = WARPS > 2 ? 2 : kWarpP;
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int p = a.p, m = a.m, G = a.G, S = a.S;
  const XT *Xp = reinterpret_cast<const XT *>(a.Xp);
  unsigned char *rows = smem;
  RowC<CT> *cst = reinterpret_cast<RowC<CT> *>(smem + P.off_consts);
  CT *dv = reinterpret_cast<CT *>(smem + P.off_d);
  CT *rho0 = reinterpret_cast<CT *>(smem + P.off_vec);  // [CPL] initial momentum
  CT *red = reinterpret_cast<CT *>(smem + P.off_red);            // [2][WARPS][2*CPL]
  double *redd = reinterpret_cast<double *>(smem + P.off_redd);  // [2][WARPS][2]
  double *blks = reinterpret_cast<double *>(smem + P.off_blk);   // [G][2]
  CT *Cs = reinterpret_cast<CT *>(smem + P.off_mat);  // [CPL, CPL] zero-padded
  CT *Sgs = Cs + CPL * CPL;                            // [CPL, CPL] zero-padded
  ResK<CT> *ks = reinterpret_cast<ResK<CT> *>(smem + P.off_k);
  const CT inv_s2 = (CT)a.inv_s2;
  const int fam = a.fam;
  const int cv1 = a.cv_order == 1;
  // per-lane column constants (slot h of lane l is column l + 32 h)
  bool col[NC];
  int cl[NC];  // the column's index into the [CPL, CPL] tiles (0 past CPL: a padded read)
  CT Bc[NC], muc[NC], ivc[NC], tbc[NC];
#pragma unroll
  for (int h = 0; h < NC; ++h) {
    const int c = lane + 32 * h;
    col[h] = c < p;
    cl[h] = c < CPL ? c : 0;
    Bc[h] = col[h] ? ldg_ct<CT>(a.B_ct, c) : CT(0);
    muc[h] = col[h] ? ldg_ct<CT>(a.mu_ct, c) : CT(0);
    ivc[h] = col[h] ? ldg_ct<CT>(a.ivar_ct, c) : CT(0);
    tbc[h] = col[h] ? ldg_ct<CT>(a.tb_ct, c) : CT(0);
  }
  const int nvec = round16(p * (int)sizeof(XT)) / 16;  // 16-byte vectors of this problem's rows

  __syncthreads();  // the previous particle is finished with shared memory
  if (reload) {
    if (tid == 0) {
      ResK<CT> k;
      k.temp = a.st->a;
      k.nm = (double)a.n / (double)m;
      k.inv_m = 1.0 / (double)m;
      k.ta = (CT)k.temp;
      k.ta2 = (CT)(k.temp * k.temp * k.nm * k.nm);
      k.tnm = (CT)(k.temp * k.nm);
      k.smv = stage_move(a.stage_dev ? a.st->stage : a.stage, a.move);
      *ks = k;
    }
    for (int e = tid; e < CPL * CPL; e += blockDim.x) {
      const int r = e / CPL, c = e - r * CPL;
      const bool in = r < p && c < p;
      Cs[e] = in ? ldg_ct<CT>(a.C_ct, r * p + c) : CT(0);
      Sgs[e] = in ? ldg_ct<CT>(a.Sigma_ct, r * p + c) : CT(0);
    }
  }
  {
    const int32_t *u = a.u + (int64_t)i * m;
    // 1. gather x_{u_j} and the row's constants at the centre (its tail) with 16-byte copies;
    // invalid indices are flagged and their rows zeroed. Vectors the tile reads beyond the row's
    // covariates (a tile wider than p) are zero-filled. The indices are staged in shared memory
    // first (the block-sum buffer is free until the last pass), so no copy waits on a global load.
    int32_t *us = reinterpret_cast<int32_t *>(dv);
    for (int j = tid; j < m; j += blockDim.x) cp_async4(us + j, u + j);
    cp_async_wait_all();
    __syncthreads();
    constexpr int NTV = (int)sizeof(RowC<CT>) / 16;
    const int nvr = P.nvl + NTV;
    // copy t = j nvr + q (vector q of row j); each thread steps by blockDim.x = dj nvr + dq
    const int dj = (int)blockDim.x / nvr, dq = (int)blockDim.x - dj * nvr;
    int j = tid / nvr, q = tid - (tid / nvr) * nvr;
    while (j < m) {
      const int k = us[j];
      unsigned char *dst = q < P.nvl ? rows + (size_t)j * P.rb + 16 * q
                                     : reinterpret_cast<unsigned char *>(cst + j) + 16 * (q - P.nvl);
      const int qs = q < P.nvl ? q : nvec + (q - P.nvl);  // 16-byte vector of the packed row
      if (k < 0 || (int64_t)k >= a.n || (q >= nvec && q < P.nvl)) {
        *reinterpret_cast<uint4 *>(dst) = make_uint4(0u, 0u, 0u, 0u);
        if (q == 0 && (k < 0 || (int64_t)k >= a.n)) set_err(a.st, kErrIndex);
      } else {
        cp_async16(dst, reinterpret_cast<const unsigned char *>(Xp + (int64_t)k * S) + 16 * qs);
      }
      j += dj;
      q += dq;
      if (q >= nvr) {
        q -= nvr;
        ++j;
      }
    }
    cp_async_wait_all();
    const ResK<CT> kc = *ks;  // written before the index-staging barrier
    const double temp = kc.temp, nm = kc.nm, inv_m = kc.inv_m;
    const CT ta = kc.ta, ta2 = kc.ta2, tnm = kc.tnm;
    const uint32_t smv = kc.smv;
    // 2. initial momentum rho = Linv' z (warp 0; shared with the other warps below)
    CT *thg = reinterpret_cast<CT *>(a.theta_out) + (int64_t)i * p;
    const CT eps = (CT)jittered_eps(a.st->eps, a.eps_jitter, a.seed, smv, (uint32_t)i);
    if (warp == 0) {
      const Stream smom(a.seed, kMomentum, smv, (uint32_t)i);
      CT z[NC], acc[NC];
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        z[h] = col[h] ? stream_normal_ct<CT>(smom, (uint32_t)(lane + 32 * h)) : CT(0);
        acc[h] = CT(0);
      }
#pragma unroll
      for (int hz = 0; hz < NC; ++hz)  // rho_r = sum_{c >= r} Linv[c, r] z_c, c ascending
        for (int cc = 0; cc < 32 && 32 * hz + cc < p; ++cc) {
          const int c = 32 * hz + cc;
          const CT zc = __shfl_sync(0xffffffffu, z[hz], cc);
#pragma unroll
          for (int h = 0; h < NC; ++h) {
            const int r = lane + 32 * h;
            if (col[h] && c >= r) acc[h] = fma(ldg_ct<CT>(a.Linv_ct, c * p + r), zc, acc[h]);
          }
        }
#pragma unroll
      for (int h = 0; h < NC; ++h)
        if (lane + 32 * h < CPL) rho0[lane + 32 * h] = col[h] ? acc[h] : CT(0);
    }
    __syncthreads();
    // every warp now carries the trajectory in its lanes: theta_c, rho_c, grad_c at lane c mod 32
    CT th[NC], rho[NC], gr[NC];
#pragma unroll
    for (int h = 0; h < NC; ++h) {
      const int c = lane + 32 * h;
      th[h] = col[h] ? thg[c] : CT(0);
      rho[h] = c < CPL ? rho0[c] : CT(0);
      gr[h] = CT(0);
    }
    CT dr[CPL];
    auto set_delta = [&]() {
      CT dl[NC];
#pragma unroll
      for (int h = 0; h < NC; ++h) dl[h] = col[h] ? th[h] - tbc[h] : CT(0);
#pragma unroll
      for (int s = 0; s < CPL; ++s) dr[s] = __shfl_sync(0xffffffffu, dl[s / 32], s % 32);
    };
    auto sigma_rho = [&](CT *vs) {  // (Sigma rho)_c at the lane's columns
#pragma unroll
      for (int h = 0; h < NC; ++h) vs[h] = CT(0);
#pragma unroll
      for (int k = 0; k < CPL; ++k) {
        const CT rk = __shfl_sync(0xffffffffu, rho[k / 32], k % 32);
#pragma unroll
        for (int h = 0; h < NC; ++h) vs[h] = fma(Sgs[k * CPL + cl[h]], rk, vs[h]);
      }
    };
    auto kinetic = [&]() -> double {  // rho' Sigma rho / 2 (every lane of the warp)
      CT v[NC];
      sigma_rho(v);
      double t = 0.0;
#pragma unroll
      for (int h = 0; h < NC; ++h) t += col[h] ? (double)rho[h] * (double)v[h] : 0.0;
      return 0.5 * warp_sum(t);
    };
    auto log_prior = [&]() -> double {
      double t = 0.0;
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        const double rr = (double)th[h] - (double)muc[h];
        t += col[h] ? -0.5 * rr * rr * (double)ivc[h] : 0.0;
      }
      return warp_sum(t) + a.log_prior_const;
    };
    set_delta();
    double ell = 0.0, sig = 0.0;
    int buf = 0;
    // shift of the row sums (identical in every warp): the cached subsample mean of d at this
    // particle's current theta and u
    CT Ksh = CT(0);
    if (a.blk) {
      const double *bc = a.blk + (int64_t)i * G * 2;
      double s0 = 0.0;
      for (int g = lane; g < G; g += 32) s0 += bc[2 * g];
      Ksh = (CT)(warp_sum(s0) * inv_m);
      if (!isfinite(Ksh)) Ksh = CT(0);
    }
    // One estimator pass at the current delta (dr). Every warp ends with the gradient at its lanes
    // and l_hat, sigma2_hat; FINAL also fills the block sums blks.
    auto pass = [&](bool final, bool want_totals) {
      CT v[2 * CPL];
#pragma unroll
      for (int s = 0; s < 2 * CPL; ++s) v[s] = CT(0);
      CT sd = CT(0), sd2 = CT(0);
      // the row loop, specialised per family (the dispatch is taken once per pass, not per row)
      auto row_loop = [&](auto famc) {
        constexpr int F = decltype(famc)::value;
        for (int j = warp * 32 + lane; j < m; j += WARPS * 32) {
          CT x[CPL];
          load_res_row<XT, CPL>(rows + (size_t)j * P.rb, x);
          const CT D = dot_slots<CPL>(x, dr);
          const RowC<CT> c = cst[j];
          CT d, r;
          row_incr<F, CT>(c, D, inv_s2, d, r);
          if (cv1) to_first_order(row_l2<F, CT>(c, inv_s2), D, d, r);
          const CT e = d - Ksh;
          axpy_slots<CPL>(r, x, v);
          axpy_slots<CPL>(e * r, x, v + CPL);
          sd += e;
          sd2 = fma(e, e, sd2);
          if (final) dv[j] = e;
        }
      };
      switch (fam) {
        case 0: row_loop(std::integral_constant<int, 0>{}); break;
        case 1: row_loop(std::integral_constant<int, 1>{}); break;
        case 2: row_loop(std::integral_constant<int, 2>{}); break;
        case 3: row_loop(std::integral_constant<int, 3>{}); break;
        default: row_loop(std::integral_constant<int, 4>{}); break;
      }
      int base = 0;
      reduce_scatter<2 * CPL, 16, CT>(v, lane, base);
      constexpr int KF = kfinal<2 * CPL, 16>();
      CT *rb = red + buf * WARPS * 2 * CPL;
      CT *rd = reinterpret_cast<CT *>(redd) + buf * WARPS * 2;
#pragma unroll
      for (int q = 0; q < KF; ++q) rb[warp * 2 * CPL + base + q] = v[q];
      const CT s1 = warp_sum(sd), s2 = warp_sum(sd2);
      if (lane == 0) {
        rd[2 * warp] = s1;
        rd[2 * warp + 1] = s2;
      }
      __syncthreads();  // all warps' partial sums of this pass are in buffer buf
      CT S1f = CT(0);   // sum of e over the subsample (the gradient needs only its mean)
#pragma unroll
      for (int w = 0; w < WARPS; ++w) S1f += rd[2 * w];
      if (final) {  // shifted block sums of e (floor partition of u into G blocks)
        for (int g = warp; g < G; g += WARPS) {
          const int j0 = (int)(((int64_t)g * m) / G), j1 = (int)(((int64_t)(g + 1) * m) / G);
          CT bs = CT(0), bq = CT(0);
          for (int j = j0 + lane; j < j1; j += 32) {
            const CT dj = dv[j];
            bs += dj;
            bq = fma(dj, dj, bq);
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
      // gradient of a l_hat - a^2/2 sigma2_hat + log p(theta) at the lane's columns (every warp)
      const CT dbar = S1f * (CT)inv_m;  // mean of e
      CT cd[NC];
#pragma unroll
      for (int h = 0; h < NC; ++h) cd[h] = CT(0);
#pragma unroll
      for (int k = 0; k < CPL; ++k)
#pragma unroll
        for (int h = 0; h < NC; ++h) cd[h] = fma(Cs[k * CPL + cl[h]], dr[k], cd[h]);
#pragma unroll
      for (int h = 0; h < NC; ++h) {
        const int c = lane + 32 * h;
        CT G1 = CT(0), G2 = CT(0);
        if (col[h]) {
#pragma unroll
          for (int w = 0; w < WARPS; ++w) {
            G1 += rb[w * 2 * CPL + c];
            G2 += rb[w * 2 * CPL + CPL + c];
          }
        }
        gr[h] = col[h] ? ta * (Bc[h] + cd[h]) + tnm * G1 - ta2 * (G2 - dbar * G1) -
                             (th[h] - muc[h]) * ivc[h]
                       : CT(0);
      }
      if (want_totals && warp == 0) {  // l_hat and sigma2_hat in FP64 (first and last pass)
        CT ql = CT(0);
#pragma unroll
        for (int h = 0; h < NC; ++h)
          if (col[h]) ql += (th[h] - tbc[h]) * (Bc[h] + CT(0.5) * cd[h]);
        const CT qlin = warp_sum(ql);
        double S1 = 0.0, S2 = 0.0;
        if (final) {
          for (int g = 0; g < G; ++g) {
            S1 += blks[2 * g];
            S2 += blks[2 * g + 1];
          }
        } else {
#pragma unroll
          for (int w = 0; w < WARPS; ++w) {
            S1 += (double)rd[2 * w];
            S2 += (double)rd[2 * w + 1];
          }
        }
        ell = (a.A_dev ? __ldg(a.A_dev) : a.A) + (double)qlin + nm * fma((double)m, (double)Ksh, S1);
        sig = nm * nm * fmax(0.0, S2 - S1 * S1 * inv_m);
      }
      if (!final) Ksh += dbar;  // the next pass is shifted by this pass's mean of d
      buf ^= 1;
    };

    // 3. trajectory. The Hamiltonian's FP64 terms (slow on this part: a warp-wide FP64
    // instruction holds the sub-partition's FP64 pipe for tens of cycles) are split over warps
    // that run on different sub-partitions: warp 0 the kinetic energy (it also assembles H and
    // runs the MH test), warp 1 the log prior, warp 2 the log of the MH uniform (fewer warps take
    // more of them); every warp carries the same theta and rho.
    double *hs = reinterpret_cast<double *>(smem + P.off_h);
    double kin0 = 0.0;
    if (warp == 0) kin0 = kinetic();
    if (warp == kWarpP) {
      const double lp = log_prior();
      if (lane == 0) hs[0] = lp;
    }
    if (warp == kWarpU && lane == 0) {
      const Stream smh(a.seed, kMhTheta, smv, (uint32_t)i);
      hs[2] = log(draw_uniform(smh.draw(0)));
    }
    pass(false, true);  // its barrier publishes hs[0] and hs[2]
    const double H0 = warp == 0 ? -(temp * ell - 0.5 * temp * temp * sig + hs[0]) + kin0 : 0.0;
    for (int l = 0; l < a.L; ++l) {
      CT vs[NC];
#pragma unroll
      for (int h = 0; h < NC; ++h) rho[h] += CT(0.5) * eps * gr[h];
      sigma_rho(vs);
#pragma unroll
      for (int h = 0; h < NC; ++h)
        if (col[h]) th[h] += eps * vs[h];
      set_delta();
      pass(l == a.L - 1, l == a.L - 1);
#pragma unroll
      for (int h = 0; h < NC; ++h) rho[h] += CT(0.5) * eps * gr[h];
    }
    // 4. Metropolis-Hastings in FP64, write-back on acceptance (warp 0)
    double kin1 = 0.0;
    if (warp == 0) kin1 = kinetic();
    if (warp == kWarpP) {
      const double lp = log_prior();
      if (lane == 0) hs[1] = lp;
    }
    __syncthreads();
    if (warp == 0) {
      const double H1 = -(temp * ell - 0.5 * temp * temp * sig + hs[1]) + kin1;
      const bool acc = hs[2] < H0 - H1;  // log U < H0 - H1; false when H1 is NaN
      if (acc) {
#pragma unroll
        for (int h = 0; h < NC; ++h)
          if (col[h]) thg[lane + 32 * h] = th[h];
        // the cache holds FP64 (sum d, sum d^2) per block: rebuilt from the shifted sums
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
}

template <typename XT, int CPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_hmc_res(EstArgs a, ResPlan P) {
  for (int il = blockIdx.x; il < a.B; il += gridDim.x)
    res_particle<XT, CPL, WARPS>(a, a.i0 + il, il == (int)blockIdx.x, P);
}

// All particles of a batch of independent posteriors (the problems of one resident tile): the
// global particle index picks the problem from the prefix offsets; the shared-memory plan is the
// largest over those problems.
template <typename XT, int CPL, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) k_hmc_res_batch(BatchArgs b, ResPlan P) {
  int qcur = -1;
  for (int g = blockIdx.x; g < b.total; g += gridDim.x) {
    const int q = batch_problem(b.offsets, b.nprob, g);
    res_particle<XT, CPL, WARPS>(b.probs[q], g - b.offsets[q], q != qcur, P);
    qcur = q;
  }
}

// dry: only check that the plan fits (no launch).
template <typename XT, int CPL, int WARPS>
inline int launch_res(const EstArgs &a, cudaStream_t s, int sms, bool dry) {
  using CT = typename Store<XT>::CT;
  if (a.p > CPL) return -2;
  const ResPlan P = res_plan<CT>(a.p, a.m, a.G, (int)sizeof(XT), WARPS, CPL);
  cudaError_t e = cudaFuncSetAttribute(k_hmc_res<XT, CPL, WARPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, P.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hmc_res<XT, CPL, WARPS>,
                                                    WARPS * 32, P.total);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return -2;
  }
  if (dry || a.B <= 0) return 0;
  const int grid = a.B < per_sm * sms ? a.B : per_sm * sms;
  k_hmc_res<XT, CPL, WARPS><<<grid, WARPS * 32, P.total, s>>>(a, P);
  return (int)cudaGetLastError();
}

// Batched launch over the problems in b (their largest p, m and G size the plan). dry: check the
// fit only. Returns a cudaError_t or -2 when the plan does not fit.
template <typename XT, int CPL, int WARPS>
inline int launch_res_batch(const BatchArgs &b, int p_max, int m_max, int G_max, cudaStream_t s,
                            int sms, bool dry) {
  using CT = typename Store<XT>::CT;
  if (p_max > CPL) return -2;
  const ResPlan P = res_plan<CT>(p_max, m_max, G_max, (int)sizeof(XT), WARPS, CPL);
  cudaError_t e = cudaFuncSetAttribute(k_hmc_res_batch<XT, CPL, WARPS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, P.total);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return -2;
  }
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hmc_res_batch<XT, CPL, WARPS>,
                                                    WARPS * 32, P.total);
  if (e != cudaSuccess || per_sm < 1) {
    cudaGetLastError();
    return -2;
  }
  if (dry || b.total <= 0) return 0;
  const int grid = b.total < per_sm * sms ? b.total : per_sm * sms;
  k_hmc_res_batch<XT, CPL, WARPS><<<grid, WARPS * 32, P.total, s>>>(b, P);
  return (int)cudaGetLastError();
}

}  // namespace subsmc
