// Device building blocks for the subsampling-SMC kernels: counter-based random numbers, the GLM
// per-row terms in increment form, storage traits of the packed row layout, warp reductions.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace subsmc {

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds, two 32x32->64 multiplies per
// round, key bumped by the Weyl increments between rounds. Stream layout used by the whole library:
// counter (draw/2, particle, stage*256 + move, tag), key (seed_lo, seed_hi); the j-th 64-bit draw of
// a stream is word pair (2h+1, 2h) of block j/2, h = j & 1.
// ------------------------------------------------------------------------------------------------
enum Tag : uint32_t {
  kInitTheta = 1, kInitU = 2, kUpmBlock = 3, kUpmIdx = 4,
  kMomentum = 5, kMhTheta = 6, kMhU = 7, kResample = 8
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

struct Stream {
  uint2 key;
  uint32_t particle, stage_move, tag;
  __device__ __forceinline__ Stream(uint64_t seed, uint32_t tag_, uint32_t sm, uint32_t i)
      : key(make_uint2((uint32_t)seed, (uint32_t)(seed >> 32))), particle(i), stage_move(sm),
        tag(tag_) {}
  // Both 64-bit draws of Philox block b: draws 2b and 2b+1.
  __device__ __forceinline__ void pair(uint32_t b, uint64_t &r0, uint64_t &r1) const {
    uint4 o = philox4x32_10(make_uint4(b, particle, stage_move, tag), key);
    r0 = ((uint64_t)o.y << 32) | o.x;
    r1 = ((uint64_t)o.w << 32) | o.z;
  }
  __device__ __forceinline__ uint64_t draw(uint64_t j) const {
    uint64_t r0, r1;
    pair((uint32_t)(j >> 1), r0, r1);
    return (j & 1) ? r1 : r0;
  }
};

__device__ __forceinline__ uint32_t stage_move(int stage, int move) {
  return ((uint32_t)stage << 8) | (uint32_t)(move & 0xFF);
}
// Index uniform on {0..n-1}: floor(r * n / 2^64).
__device__ __forceinline__ int64_t draw_index(uint64_t r, uint64_t n) {
  return (int64_t)__umul64hi(r, n);
}
__device__ __forceinline__ double draw_uniform(uint64_t r) {
  return (double)(r >> 11) * 0x1.0p-53;
}
// Particle i's HMC step size: eps times a uniform on [1 - jitter, 1 + jitter] taken from the
// second 64-bit word of its theta-MH block (the first is the MH uniform). A random step size
// breaks the near-periodic trajectories that a fixed eps L gives on near-Gaussian targets.
__device__ __forceinline__ double jittered_eps(double eps, double jitter, uint64_t seed,
                                               uint32_t sm, uint32_t i) {
  if (!(jitter > 0.0)) return eps;
  const double U = draw_uniform(Stream(seed, kMhTheta, sm, i).draw(1));
  return eps * (1.0 - jitter + 2.0 * jitter * U);
}

// Box-Muller (1958) on one Philox block: u1 in (0,1], u2 in [0,1).
__device__ __forceinline__ void box_muller(uint64_t ra, uint64_t rb, double &z0, double &z1) {
  const double u1 = (double)((ra >> 11) + 1) * 0x1.0p-53;
  const double u2 = (double)(rb >> 11) * 0x1.0p-53;
  const double r = sqrt(-2.0 * log(u1));
  double s, c;
  sincospi(2.0 * u2, &s, &c);
  z0 = r * c;
  z1 = r * s;
}
__device__ __forceinline__ double stream_normal(const Stream &st, uint32_t j) {
  uint64_t ra, rb;
  st.pair(j >> 1, ra, rb);
  double z0, z1;
  box_muller(ra, rb, z0, z1);
  return (j & 1) ? z1 : z0;
}
// The same normal evaluated in FP32 (for FP32 particle states): the same u1 = (k + 1) 2^-53 and
// u2, with log u1 formed without losing the integer's bits: logf of the exactly scaled value when
// u1 < 1/2, log1pf of the exact integer complement -(2^53 - 1 - k) 2^-53 otherwise. Agrees with
// the FP64 value rounded to FP32 to a few units in the last place.
__device__ __forceinline__ float stream_normal_f32(const Stream &st, uint32_t j) {
  uint64_t ra, rb;
  st.pair(j >> 1, ra, rb);
  const uint64_t k = ra >> 11;
  const float lu = k < (1ull << 52) ? logf((float)(k + 1) * 0x1.0p-53f)
                                    : log1pf(-(float)((1ull << 53) - 1 - k) * 0x1.0p-53f);
  const float r = sqrtf(-2.0f * lu);
  float sn, cs;
  sincospif(2.0f * ((float)(rb >> 11) * 0x1.0p-53f), &sn, &cs);
  return (j & 1) ? r * sn : r * cs;
}
template <typename CT> __device__ __forceinline__ CT stream_normal_ct(const Stream &st, uint32_t j) {
  if constexpr (sizeof(CT) == 4)
    return stream_normal_f32(st, j);
  else
    return stream_normal(st, j);
}

// ------------------------------------------------------------------------------------------------
// Packed row layout. Row k of the library's copy of the data holds
//   [x_k1 .. x_kp | zeros to a 16-byte boundary | RowC tail {c0, c1, c2, y_k} | zeros]
// with x from element 0 (every row and its covariates start 16-byte aligned), the tail at element
// Yo in the state type (16 bytes; 32 for FP64) and the row stride S a multiple of 64 bytes, so a
// gathered row occupies whole DRAM fetch units. c0..c2 are the trajectory-invariant constants of
// the row at the control-variate centre (row_consts below); they are rewritten whenever the centre
// changes.
// ------------------------------------------------------------------------------------------------
template <typename XT> struct Store;
template <> struct Store<double> {
  using CT = double;  // arithmetic type of the per-row terms
  static constexpr int VEC = 2;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    out[0] = __hiloint2double((int)v.y, (int)v.x);
    out[1] = __hiloint2double((int)v.w, (int)v.z);
  }
};
template <> struct Store<float> {
  using CT = float;
  static constexpr int VEC = 4;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    out[0] = __uint_as_float(v.x);
    out[1] = __uint_as_float(v.y);
    out[2] = __uint_as_float(v.z);
    out[3] = __uint_as_float(v.w);
  }
};
template <> struct Store<__nv_bfloat16> {
  using CT = float;
  static constexpr int VEC = 8;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      out[2 * q] = __uint_as_float(w[q] << 16);
      out[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
};

// ------------------------------------------------------------------------------------------------
// GLM per-row terms in increment form. With eta_bar = x'theta_bar and D = x'(theta - theta_bar):
//   d = l(eta_bar + D) - [l(eta_bar) + l'(eta_bar) D + l''(eta_bar) D^2 / 2]   (l_k - q_k, Sec. 3.2)
//   r = l'(eta_bar + D) - l'(eta_bar) - l''(eta_bar) D                     (d/d eta of d)
// The forms below are algebraically equal to these definitions but are arranged so that rounding
// error scales with |D| rather than with |l|: the second-order expansion cancels analytically.
// ------------------------------------------------------------------------------------------------
template <typename CT> __device__ __forceinline__ CT softplus_(CT x) {
  return x > CT(0) ? x + log1p(exp(-x)) : log1p(exp(x));
}
template <typename CT> __device__ __forceinline__ CT sigmoid_(CT x) {
  return x >= CT(0) ? CT(1) / (CT(1) + exp(-x)) : exp(x) / (CT(1) + exp(x));
}

// e^D - 1 - D - D^2/2 (k0 = 3) or e^D - 1 - D (k0 = 2) by the Taylor series of exp for |D| <= 1
// (FP32; 1/2 in FP64), directly from expm1 otherwise.
template <typename CT, int K0> __device__ __forceinline__ CT exp_tail(CT D) {
  constexpr CT kMax = sizeof(CT) == 8 ? CT(0.5) : CT(1);
  if (fabs(D) <= kMax) {
    // terms k0 .. k0+NT-1: the remainder is below 1e-17 (FP64, |D| <= 1/2) or 1e-9 (FP32,
    // |D| <= 1) relative to the first term
    constexpr int NT = sizeof(CT) == 8 ? 19 : 10;
    // s = sum_{j>=0} D^j k0!/(k0+j)!, by Horner with the constant reciprocals 1/k
    CT s = CT(1);
#pragma unroll
    for (int k = K0 + NT - 1; k > K0; --k) s = fma(s * D, CT(1.0 / k), CT(1));
    constexpr double inv_f = K0 == 2 ? 0.5 : 1.0 / 6.0;  // 1/k0!
    CT Dk = D;
#pragma unroll
    for (int k = 1; k < K0; ++k) Dk *= D;
    return Dk * CT(inv_f) * s;
  }
  CT t = expm1(D) - D;
  if (K0 == 3) t -= CT(0.5) * D * D;
  return t;
}

// log Phi(z) and lambda(z) = phi(z)/Phi(z) from CUDA's erfc/erfcx.
template <typename CT> __device__ __forceinline__ void log_phi_(CT z, CT &lp, CT &lam) {
  const CT x = -z * CT(0.70710678118654752440);
  const CT ex = erfcx(x);
  lam = CT(0.79788456080286535588) / ex;
  if (z < CT(0))
    lp = log(CT(0.5) * ex) - x * x;
  else
    lp = log1p(CT(-0.5) * erfc(-x));
}

// Trajectory-invariant per-row constants: they depend on eta_bar = x'theta_bar and y only, so they
// are computed once per centre and stored in the row's tail; row_incr(row_consts(...)) gives d, r.
//   logistic: c0 = sigma(eta_bar), c1 = c0 (1 - c0), c2 = eta_bar
//   Poisson:  c0 = e^eta_bar
//   Gaussian: c0 = y - eta_bar
//   probit:   c0 = z_bar = s eta_bar (s = 2y - 1), c1 = log Phi(z_bar), c2 = lambda(z_bar)
//   Student-t: c0 = r_bar = y - eta_bar, c1 = 1 / (nu s^2 + r_bar^2), c2 = nu + 1
template <typename CT> struct alignas(16) RowC {
  CT c0, c1, c2, y;
};

// nu: degrees of freedom of the Student-t family (unused by the others).
template <int FAM, typename CT>
__device__ __forceinline__ RowC<CT> row_consts(CT eb, CT y, CT inv_s2, CT nu = CT(0)) {
  RowC<CT> c;
  c.c0 = c.c1 = c.c2 = CT(0);
  c.y = y;
  if (FAM == 4) {
    const CT rb = y - eb;
    c.c0 = rb;
    c.c1 = CT(1) / fma(rb, rb, nu / inv_s2);
    c.c2 = nu + CT(1);
  } else if (FAM == 0) {
    const CT sb = sigmoid_(eb);
    c.c0 = sb;
    c.c1 = sb * (CT(1) - sb);
    c.c2 = eb;
  } else if (FAM == 2) {
    c.c0 = exp(eb);
  } else if (FAM == 3) {
    c.c0 = y - eb;
  } else {
    const CT zb = (CT(2) * y - CT(1)) * eb;
    CT lpb, lamb;
    log_phi_(zb, lpb, lamb);
    c.c0 = zb;
    c.c1 = lpb;
    c.c2 = lamb;
  }
  (void)inv_s2;
  return c;
}

// Horner steps of the two cumulant-series chains at once (FP32: one packed FMA per step):
// (pd, pr) = (pd, pr) * D + kappa * (1/k!, 1/(k-1)!).
template <typename CT>
__device__ __forceinline__ void horner2(CT &pd, CT &pr, CT D, CT kappa, double fd, double fr) {
  pd = fma(pd, D, kappa * CT(fd));
  pr = fma(pr, D, kappa * CT(fr));
}
template <>
__device__ __forceinline__ void horner2<float>(float &pd, float &pr, float D, float kappa,
                                               double fd, double fr) {
  const float2 coef = __fmul2_rn(make_float2(kappa, kappa), make_float2((float)fd, (float)fr));
  const float2 v = __ffma2_rn(make_float2(pd, pr), make_float2(D, D), coef);
  pd = v.x;
  pr = v.y;
}

// short4: the caller has checked |D| <= 1/20 for every lane of the warp (FP32 only); the
// logistic series then stops at kappa_6 (truncation below 2e-8 of w|D|^3 and w D^2).
template <int FAM, typename CT>
__device__ __forceinline__ void row_incr(const RowC<CT> &c, CT D, CT inv_s2, CT &d, CT &r,
                                         bool short4 = false) {
  if (FAM == 0) {  // logistic: l = y*eta - log(1 + e^eta); y cancels from d and r
    const CT sb = c.c0, w = c.c1;
    // With K(D) = log(1 - s + s e^D), the cumulant generating function of Bernoulli(s), s = sigma(eta_bar):
    //   d = -(K(D) - s D - w D^2/2) = -sum_{k>=3} kappa_k D^k / k!,  r = -sum_{k>=3} kappa_k D^(k-1) / (k-1)!
    // kappa_3..kappa_10 are polynomials in w = s(1-s) and q = 1 - 2s (kappa_{k+1} = w d kappa_k/ds).
    // The series converges for |D| < pi; up to |D| = 1/2 (1/20 in FP64) terms to kappa_10 leave a
    // relative error below 1e-8 in d and 1e-7 in r (1e-15 in FP64). No transcendental, no
    // division, no cancellation.
    constexpr CT kSmall = sizeof(CT) == 8 ? CT(0.05) : CT(0.5);
    if (sizeof(CT) == 4 && short4) {
      const CT q = CT(1) - CT(2) * sb;
      const CT k3 = w * q;
      const CT k4 = w * (CT(1) - CT(6) * w);
      const CT k5 = k3 * (CT(1) - CT(12) * w);
      const CT k6 = w * (CT(1) + w * (CT(-30) + CT(120) * w));
      CT pd = k6 * CT(1.0 / 720.0), pr = k6 * CT(1.0 / 120.0);
      horner2(pd, pr, D, k5, 1.0 / 120.0, 1.0 / 24.0);
      horner2(pd, pr, D, k4, 1.0 / 24.0, 1.0 / 6.0);
      horner2(pd, pr, D, k3, 1.0 / 6.0, 0.5);
      const CT D2 = D * D;
      d = -D2 * D * pd;
      r = -D2 * pr;
      return;
    }
    // FP32: one form per warp (a vote over the lanes evaluating a row here), so a warp whose rows
    // straddle |D| = 1/2 does not run both forms; rows with small |D| in a warp that takes the
    // exp/log form carry that form's absolute error (about 3e-7) instead of the series' relative one
    bool series;
    if constexpr (sizeof(CT) == 4)
      series = !__any_sync(__activemask(), fabs(D) > kSmall);
    else
      series = fabs(D) <= kSmall;
    if (series) {
      const CT q = CT(1) - CT(2) * sb;
      const CT k3 = w * q;
      const CT k4 = w * (CT(1) - CT(6) * w);
      const CT k5 = k3 * (CT(1) - CT(12) * w);
      const CT k6 = w * (CT(1) + w * (CT(-30) + CT(120) * w));
      const CT k7 = k3 * (CT(1) + w * (CT(-60) + CT(360) * w));
      const CT k8 = w * (CT(1) + w * (CT(-126) + w * (CT(1680) - CT(5040) * w)));
      const CT k9 = k3 * (CT(1) + w * (CT(-252) + w * (CT(5040) - CT(20160) * w)));
      const CT k10 =
          w * (CT(1) + w * (CT(-510) + w * (CT(17640) + w * (CT(-151200) + CT(362880) * w))));
      CT pd = k10 * CT(1.0 / 3628800.0), pr = k10 * CT(1.0 / 362880.0);
      horner2(pd, pr, D, k9, 1.0 / 362880.0, 1.0 / 40320.0);
      horner2(pd, pr, D, k8, 1.0 / 40320.0, 1.0 / 5040.0);
      horner2(pd, pr, D, k7, 1.0 / 5040.0, 1.0 / 720.0);
      horner2(pd, pr, D, k6, 1.0 / 720.0, 1.0 / 120.0);
      horner2(pd, pr, D, k5, 1.0 / 120.0, 1.0 / 24.0);
      horner2(pd, pr, D, k4, 1.0 / 24.0, 1.0 / 6.0);
      horner2(pd, pr, D, k3, 1.0 / 6.0, 0.5);
      const CT D2 = D * D;
      d = -D2 * D * pd;
      r = -D2 * pr;
      return;
    }
    if constexpr (sizeof(CT) == 4) {
      // |D| > 1/2 in FP32: with eta = eta_bar + D and softplus(x) = max(x, 0) + log(1 + e^-|x|),
      //   L1 = softplus(eta) - softplus(eta_bar)
      //      = [max(eta, 0) - max(eta_bar, 0)] + log(1 + e^-|eta|) - log(1 + e^-|eta_bar|),
      // where log(1 + e^-|eta_bar|) = -log(max(s, 1 - s)) (1 - s is exact for s >= 1/2), and
      // sigma(eta) = 1/(1 + e^-|eta|) for eta >= 0, e^-|eta|/(1 + e^-|eta|) otherwise: one
      // exponential, two logarithms and one reciprocal, no overflow for any eta. The hardware
      // approximations (MUFU ex2/lg2/rcp) err by about 2e-7 absolute, the size of what d loses
      // to its own cancellation (-L1 + sD + wD^2/2) at this |D| in FP32 anyway.
      const float eb = c.c2, eta = eb + D;
      const float e = __expf(-fabsf(eta)), ope = 1.0f + e;
      const float lb = __logf(fmaxf(sb, 1.0f - sb));
      const float pos = eb >= 0.0f ? (eta >= 0.0f ? D : -eb) : (eta >= 0.0f ? eta : 0.0f);
      const float L1f = pos + (__logf(ope) + lb);
      const float inv = __fdividef(1.0f, ope);
      const float sg = eta >= 0.0f ? inv : e * inv;
      r = fmaf(w, D, sb - sg);
      d = fmaf(0.5f * w * D, D, fmaf(sb, D, -L1f));
      return;
    }
    CT L1;
    if (fabs(D) <= CT(1)) {
      const CT e = expm1(D), t = CT(1) + sb * e;
      L1 = log1p(sb * e);  // softplus(eb + D) - softplus(eb)
      r = w * (D - e / t);
    } else {
      const CT eb = c.c2;
      L1 = softplus_(eb + D) - softplus_(eb);
      r = sb - sigmoid_(eb + D) + w * D;
    }
    d = -L1 + sb * D + CT(0.5) * w * D * D;
  } else if (FAM == 4) {  // Student-t: l = const - (nu+1)/2 log(nu s^2 + (y - eta)^2)
    // With r = r_bar - D, q = nu s^2 + r^2 = q_bar (1 + w), w = (D^2 - 2 r_bar D) b, b = 1/q_bar:
    //   l - l_bar = -(nu+1)/2 log1p(w); its first two Taylor terms in D are -(nu+1)/2 (a D +
    //   (b - a^2/2) D^2) with a = -2 r_bar b, so
    //   d = -(nu+1)/2 [L3(w) - a b D^3 - b^2 D^4 / 2],  L3(w) = log1p(w) - w + w^2/2,
    //   r = -(nu+1) b^2 D^2 [r_bar (3 - 4 r_bar^2 b) + (2 r_bar^2 b - 1) D] / (1 + w),
    // both free of the cancellation of the printed definitions. L3 = w^3 sum_j (-w)^j / (j + 3)
    // by its series for small |w| (terms w^3 .. w^14: the remainder is below 2e-8 of w^3/3 for
    // |w| <= 1/4 in FP32, below 1e-16 for |w| <= 1/20 in FP64), else directly.
    const CT rb = c.c0, b = c.c1, nu1 = c.c2;
    const CT w = (D * D - CT(2) * rb * D) * b;
    constexpr CT kSmall = sizeof(CT) == 8 ? CT(0.05) : CT(0.25);
    CT L3;
    if (fabs(w) <= kSmall) {
      CT s = CT(1.0 / 14.0);
#pragma unroll
      for (int k = 13; k >= 3; --k) s = fma(s, -w, CT(1.0 / k));
      L3 = w * w * w * s;
    } else {
      L3 = log1p(w) - w + CT(0.5) * w * w;
    }
    const CT a = CT(-2) * rb * b, D2 = D * D;
    d = CT(-0.5) * nu1 * (L3 - a * b * D2 * D - CT(0.5) * b * b * D2 * D2);
    const CT rb2b = rb * rb * b;
    r = -nu1 * b * b * D2 * fma(fma(CT(2), rb2b, CT(-1)), D, rb * (CT(3) - CT(4) * rb2b)) /
        (CT(1) + w);
  } else if (FAM == 2) {  // Poisson: d = -e^eb tail3(D), r = -e^eb tail2(D)
    const CT t3 = exp_tail<CT, 3>(D);  // e^D - 1 - D - D^2/2; e^D - 1 - D = t3 + D^2/2
    d = -c.c0 * t3;
    r = -c.c0 * fma(CT(0.5) * D, D, t3);
  } else if (FAM == 3) {  // Gaussian, known sd: the expansion is exact; evaluated as written
    const CT res = c.c0;
    const CT dl = (CT(2) * res * D - D * D) * (CT(0.5) * inv_s2);  // l(eta) - l(eta_bar)
    d = dl - res * inv_s2 * D + CT(0.5) * inv_s2 * D * D;
    r = (res - D) * inv_s2 - res * inv_s2 + inv_s2 * D;
  } else {  // probit: l = log Phi(s*eta)
    const CT s = CT(2) * c.y - CT(1), zb = c.c0, lpb = c.c1, lamb = c.c2, z = zb + s * D;
    CT lp, lam;
    log_phi_(z, lp, lam);
    const CT h = lamb * (zb + lamb);  // -l''(eta_bar)
    d = lp - lpb - s * lamb * D + CT(0.5) * h * D * D;
    r = s * (lam - lamb) + h * D;
  }
}

// l''(eta_bar) of a row from its stored constants.
template <int FAM, typename CT> __device__ __forceinline__ CT row_l2(const RowC<CT> &c, CT inv_s2) {
  if (FAM == 0) return -c.c1;
  if (FAM == 2) return -c.c0;
  if (FAM == 3) return -inv_s2;
  if (FAM == 4) return c.c2 * c.c1 * fma(CT(2) * c.c0 * c.c0, c.c1, CT(-1));
  return -c.c2 * (c.c0 + c.c2);
}
// First-order control variates: d and r of the second-order forms plus the second-order term,
// d1 = d2 + l''(eta_bar) D^2 / 2, r1 = r2 + l''(eta_bar) D.
template <typename CT> __device__ __forceinline__ void to_first_order(CT l2, CT D, CT &d, CT &r) {
  d = fma(CT(0.5) * l2 * D, D, d);
  r = fma(l2, D, r);
}
__device__ __forceinline__ float row_l2_any(int fam, const RowC<float> &c, float inv_s2) {
  switch (fam) {
    case 0: return row_l2<0, float>(c, inv_s2);
    case 1: return row_l2<1, float>(c, inv_s2);
    case 2: return row_l2<2, float>(c, inv_s2);
    case 3: return row_l2<3, float>(c, inv_s2);
    default: return row_l2<4, float>(c, inv_s2);
  }
}
__device__ __forceinline__ double row_l2_any(int fam, const RowC<double> &c, double inv_s2) {
  switch (fam) {
    case 0: return row_l2<0, double>(c, inv_s2);
    case 1: return row_l2<1, double>(c, inv_s2);
    case 2: return row_l2<2, double>(c, inv_s2);
    case 3: return row_l2<3, double>(c, inv_s2);
    default: return row_l2<4, double>(c, inv_s2);
  }
}

// Full per-row value and derivatives at eta (used by the moment kernel, FP64). s2: the Gaussian
// variance or the Student-t squared scale; nu: the Student-t degrees of freedom.
template <int FAM>
__device__ __forceinline__ void row_value(double eta, double y, double s2, double nu, double &l,
                                          double &d1, double &d2) {
  if (FAM == 4) {
    const double r = y - eta, q = fma(r, r, nu * s2);
    l = lgamma(0.5 * (nu + 1.0)) - lgamma(0.5 * nu) - 0.5 * log(3.14159265358979323846 * nu * s2) -
        0.5 * (nu + 1.0) * log1p(r * r / (nu * s2));
    d1 = (nu + 1.0) * r / q;
    d2 = (nu + 1.0) * (r * r - nu * s2) / (q * q);
  } else if (FAM == 0) {
    const double s = sigmoid_(eta);
    l = y * eta - softplus_(eta);
    d1 = y - s;
    d2 = -s * (1.0 - s);
  } else if (FAM == 2) {
    const double mu = exp(eta);
    l = y * eta - mu - lgamma(y + 1.0);
    d1 = y - mu;
    d2 = -mu;
  } else if (FAM == 3) {
    const double r = y - eta;
    l = -0.5 * log(6.283185307179586476925286766559 * s2) - r * r / (2.0 * s2);
    d1 = r / s2;
    d2 = -1.0 / s2;
  } else {
    const double sg = 2.0 * y - 1.0, z = sg * eta;
    double lp, lam;
    log_phi_(z, lp, lam);
    l = lp;
    d1 = sg * lam;
    d2 = -lam * (z + lam);
  }
}

// ------------------------------------------------------------------------------------------------
// Warp reductions
// ------------------------------------------------------------------------------------------------
template <typename V> __device__ __forceinline__ V warp_sum(V v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename V> __device__ __forceinline__ V warp_max(V v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Per-lane sums over CPL element slots. FP32 uses the packed two-wide FMA of sm_100+ (__ffma2_rn:
// two independent round-to-nearest FMAs per instruction), halving the FMA instruction count.
template <int CPL>
__device__ __forceinline__ float dot_slots(const float *x, const float *y) {
  static_assert(CPL % 2 == 0, "pairs of slots");
  float2 a = make_float2(0.f, 0.f), b = make_float2(0.f, 0.f);
#pragma unroll
  for (int e = 0; e < CPL; e += 4) {
    a = __ffma2_rn(make_float2(x[e], x[e + 1]), make_float2(y[e], y[e + 1]), a);
    if (e + 2 < CPL) b = __ffma2_rn(make_float2(x[e + 2], x[e + 3]), make_float2(y[e + 2], y[e + 3]), b);
  }
  return (a.x + b.x) + (a.y + b.y);
}
template <int CPL>
__device__ __forceinline__ double dot_slots(const double *x, const double *y) {
  double a = 0.0, b = 0.0;
#pragma unroll
  for (int e = 0; e < CPL; e += 2) {
    a = fma(x[e], y[e], a);
    if (e + 1 < CPL) b = fma(x[e + 1], y[e + 1], b);
  }
  return a + b;
}
// acc[s] += t * x[s] over the slots
template <int CPL> __device__ __forceinline__ void axpy_slots(float t, const float *x, float *acc) {
  const float2 tt = make_float2(t, t);
#pragma unroll
  for (int e = 0; e < CPL; e += 2) {
    const float2 r = __ffma2_rn(tt, make_float2(x[e], x[e + 1]), make_float2(acc[e], acc[e + 1]));
    acc[e] = r.x;
    acc[e + 1] = r.y;
  }
}
template <int CPL>
__device__ __forceinline__ void axpy_slots(double t, const double *x, double *acc) {
#pragma unroll
  for (int e = 0; e < CPL; ++e) acc[e] = fma(t, x[e], acc[e]);
}

// Reduce-scatter of K values per lane over lane groups of size 2*O (recursive halving at offsets
// O, O/2, .., 1, then a butterfly while the count is odd). On return v[0..kfinal(K)) hold sums over
// the group of the original entries base + i.
template <int K, int O, typename V>
__device__ __forceinline__ void reduce_scatter(V *v, int lane, int &base) {
  if constexpr (O > 0) {
    if constexpr (K % 2 == 0) {
      constexpr int H = K / 2;
      const bool up = (lane & O) != 0;
#pragma unroll
      for (int i = 0; i < H; ++i) {
        const V send = up ? v[i] : v[i + H];
        const V keep = up ? v[i + H] : v[i];
        v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
      }
      if (up) base += H;
      reduce_scatter<H, O / 2, V>(v, lane, base);
    } else {
#pragma unroll
      for (int i = 0; i < K; ++i) v[i] += __shfl_xor_sync(0xffffffffu, v[i], O);
      reduce_scatter<K, O / 2, V>(v, lane, base);
    }
  }
}
template <int K, int O> __host__ __device__ constexpr int kfinal() {
  if constexpr (O == 0)
    return K;
  else if constexpr (K % 2 == 0)
    return kfinal<K / 2, O / 2>();
  else
    return kfinal<K, O / 2>();
}

}  // namespace subsmc
