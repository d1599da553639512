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

// ------------------------------------------------------------------------------------------------
// Packed row layout. Row k of the library's copy of the data holds [y_k | x_k1 .. x_kp | zeros],
// y in the first YS element slots, row stride S elements (a multiple of 16 bytes) so every row
// starts 16-byte aligned and can be read with 128-bit loads. Padding slots are zero.
// ------------------------------------------------------------------------------------------------
template <typename XT> struct Store;
template <> struct Store<double> {
  using CT = double;  // arithmetic type of the per-row terms
  using YT = double;
  static constexpr int YS = 1, VEC = 2;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    out[0] = __hiloint2double((int)v.y, (int)v.x);
    out[1] = __hiloint2double((int)v.w, (int)v.z);
  }
  __device__ __forceinline__ static YT y_of(const uint4 &v) {
    return __hiloint2double((int)v.y, (int)v.x);
  }
};
template <> struct Store<float> {
  using CT = float;
  using YT = float;
  static constexpr int YS = 1, VEC = 4;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    out[0] = __uint_as_float(v.x);
    out[1] = __uint_as_float(v.y);
    out[2] = __uint_as_float(v.z);
    out[3] = __uint_as_float(v.w);
  }
  __device__ __forceinline__ static YT y_of(const uint4 &v) { return __uint_as_float(v.x); }
};
template <> struct Store<__nv_bfloat16> {
  using CT = float;
  using YT = float;
  static constexpr int YS = 2, VEC = 8;
  __device__ __forceinline__ static void unpack(const uint4 &v, CT *out) {
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      out[2 * q] = __uint_as_float(w[q] << 16);
      out[2 * q + 1] = __uint_as_float(w[q] & 0xFFFF0000u);
    }
  }
  __device__ __forceinline__ static YT y_of(const uint4 &v) { return __uint_as_float(v.x); }
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

// e^D - 1 - D - D^2/2 (k0 = 3) or e^D - 1 - D (k0 = 2) by the Taylor series of exp for |D| <= 1/2,
// directly from expm1 otherwise.
template <typename CT, int K0> __device__ __forceinline__ CT exp_tail(CT D) {
  if (fabs(D) <= CT(0.5)) {
    constexpr int NT = sizeof(CT) == 8 ? 19 : 10;  // terms k0 .. k0+NT-1; remainder < ulp
    CT s = CT(1);
#pragma unroll
    for (int k = K0 + NT - 1; k > K0; --k) s = CT(1) + s * D / CT(k);
    // s = sum_{j>=0} D^j k0!/(k0+j)!
    CT f = CT(1);
#pragma unroll
    for (int k = 2; k <= K0; ++k) f *= CT(k);
    CT Dk = D;
#pragma unroll
    for (int k = 1; k < K0; ++k) Dk *= D;
    return Dk / f * s;
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

template <int FAM, typename CT>
__device__ __forceinline__ void row_terms(CT eb, CT D, CT y, CT inv_s2, CT &d, CT &r) {
  if (FAM == 0) {  // logistic: l = y*eta - log(1 + e^eta); y cancels from d and r
    const CT sb = sigmoid_(eb), w = sb * (CT(1) - sb);
    CT L1;
    if (fabs(D) <= CT(1)) {
      const CT e = expm1(D), t = CT(1) + sb * e;
      L1 = log1p(sb * e);  // softplus(eb + D) - softplus(eb)
      r = w * (D - e / t);
    } else {
      L1 = softplus_(eb + D) - softplus_(eb);
      r = sb - sigmoid_(eb + D) + w * D;
    }
    d = -L1 + sb * D + CT(0.5) * w * D * D;
  } else if (FAM == 2) {  // Poisson: l = y*eta - e^eta - log y!;  d = -e^eb tail3(D), r = -e^eb tail2(D)
    const CT mu = exp(eb);
    d = -mu * exp_tail<CT, 3>(D);
    r = -mu * exp_tail<CT, 2>(D);
  } else if (FAM == 3) {  // Gaussian, known sd: the expansion is exact; evaluated as written
    const CT res = y - eb;
    const CT dl = (CT(2) * res * D - D * D) * (CT(0.5) * inv_s2);  // l(eta) - l(eta_bar)
    d = dl - res * inv_s2 * D + CT(0.5) * inv_s2 * D * D;
    r = (res - D) * inv_s2 - res * inv_s2 + inv_s2 * D;
  } else {  // probit: l = log Phi(s*eta), s = 2y - 1
    const CT s = CT(2) * y - CT(1), zb = s * eb, z = s * (eb + D);
    CT lpb, lamb, lp, lam;
    log_phi_(zb, lpb, lamb);
    log_phi_(z, lp, lam);
    const CT h = lamb * (zb + lamb);  // -l''(eta_bar)
    d = lp - lpb - s * lamb * D + CT(0.5) * h * D * D;
    r = s * (lam - lamb) + h * D;
  }
}

// Full per-row value and derivatives at eta (used by the moment kernel, FP64).
template <int FAM>
__device__ __forceinline__ void row_value(double eta, double y, double s2, double &l, double &d1,
                                          double &d2) {
  if (FAM == 0) {
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

}  // namespace subsmc
