// Moments of the Laplace-tilted edge marginal, device side.
//
// Sec. III-C, Eq. marginal_tilted_un: for an edge (i, j) of V_k with cavity
// means m_i, m_j and variances c_i, c_j, the tilted law of u = x_i - x_j is
// N(u; mu, s^2) exp(-lam |u|), mu = m_i - m_j, s^2 = c_i + c_j.  It splits into
// two Gaussians truncated at zero.  In standard units z = mu / s, l = lam * s,
// a+ = l - z, a- = l + z, the weight of the u >= 0 half is
//     w+ = erfcx(a+/sqrt2) / (erfcx(a+/sqrt2) + erfcx(a-/sqrt2)),
// and with the inverse Mills ratio h(a) = sqrt(2/pi) / erfcx(a/sqrt2),
// g(a) = h(a) - a and v(a) = 1 - h(a) g(a) the halves have
//     E+ / s = g(a+),  E- / s = -g(a-),  V+- / s^2 = v(a+-).
// The site update needs four numbers, each formed from its own formula so that
// it keeps its relative accuracy where it is small:
//     d   = (ubar - mu) / s^2 = [w+ (h+ - l) - w- (h- - l)] / s
//     q   = Sbar / s^2        = w+ v+ + w- v- + w+ w- (g+ + g-)^2
//     rho = 1 - q             = w+ h+ g+ + w- h- g- - w+ w- (g+ + g-)^2
//     eab = E|u|              = s (w+ g+ + w- g-)
// (1 - v = h g, so rho needs no subtraction from 1; it still cancels when
// l -> 0 with both halves weighted, which is where the FP64 path takes over.)
// For a >= CF_SWITCH, g and v come from Laplace's continued fraction of the
// Mills ratio, g = t_1, v = t_1 (t_2 - t_1), t_k = k / (a + t_{k+1}).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

namespace eptv {

template <typename T> struct TiltedConst;
template <> struct TiltedConst<float> {
  // direct form below 6 (relative error of v about 40 ulp at a = 6); 10 terms of
  // the continued fraction keep g and v within 2e-7 for a >= 6
  static constexpr float cf_switch = 6.0f;
  static constexpr int cf_terms = 10;
};
template <> struct TiltedConst<double> {
  static constexpr double cf_switch = 5.0;
  static constexpr int cf_terms = 48;
};

__device__ __forceinline__ float erfcx_t(float x) { return erfcxf(x); }
__device__ __forceinline__ double erfcx_t(double x) { return erfcx(x); }

// Reciprocal and reciprocal square root: the hardware approximations in FP32
// (one rounding step each, about 1 ulp), exact IEEE operations in FP64.
__device__ __forceinline__ float rcp_t(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp_t(double x) { return 1.0 / x; }
__device__ __forceinline__ float rsqrt_t(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsqrt_t(double x) { return 1.0 / sqrt(x); }

// g(a) = h(a) - a and v(a) = 1 - h(a) g(a) for a standard normal truncated to
// [a, inf); `ex` is erfcx(a / sqrt2), already computed for the weights.
template <typename T>
__device__ __forceinline__ void mills(T a, T ex, T& h, T& g, T& v) {
  const T sqrt_2_over_pi = T(0.79788456080286535588);
  if (a < TiltedConst<T>::cf_switch) {
    h = sqrt_2_over_pi * rcp_t(ex);  // ex = inf gives h = 0 for a -> -inf
    g = h - a;
    v = T(1) - h * g;
  } else {
    T t = T(0), t2 = T(0);
#pragma unroll
    for (int k = TiltedConst<T>::cf_terms; k >= 1; --k) {
      t = T(k) * rcp_t(a + t);
      if (k == 2) t2 = t;
    }
    g = t;
    h = a + t;
    v = t * (t2 - t);
  }
}

template <typename T>
struct TiltedOut {
  T d;    // (ubar - mu) / s^2
  T q;    // Sbar / s^2
  T rho;  // 1 - Sbar / s^2
  T eab;  // E|u|
};

template <typename T>
__device__ __forceinline__ TiltedOut<T> laplace_tilted(T mu, T s2, T lam) {
  const T inv_sqrt2 = T(0.70710678118654752440);
  const T rs = rsqrt_t(s2);
  T s = s2 * rs;
  T z = mu * rs;
  T l = lam * s;
  T ap = l - z, am = l + z;
  T exp_ = erfcx_t(ap * inv_sqrt2);
  T exm = erfcx_t(am * inv_sqrt2);
  // w+ = 1 / (1 + r), w- = 1 / (1 + 1/r), r = exm / exp_; one of the two
  // erfcx values may be +inf (argument below about -9 in FP32), never both.
  T r = exm * rcp_t(exp_);
  T wp = rcp_t(T(1) + r);
  T wm = rcp_t(T(1) + rcp_t(r));
  T hp, gp, vp, hm, gm, vm;
  mills<T>(ap, exp_, hp, gp, vp);
  mills<T>(am, exm, hm, gm, vm);
  TiltedOut<T> o;
  // a weight of exactly zero must not multiply an infinite or NaN partner
  T dp = wp > T(0) ? wp * (hp - l) : T(0);
  T dm = wm > T(0) ? wm * (hm - l) : T(0);
  o.d = (dp - dm) * rs;
  T gs = gp + gm;
  T mix = wp * wm * gs * gs;
  o.q = wp * vp + wm * vm + mix;
  T hgp = wp > T(0) ? wp * hp * gp : T(0);
  T hgm = wm > T(0) ? wm * hm * gm : T(0);
  o.rho = hgp + hgm - mix;
  o.eab = s * (wp * gp + wm * gm);
  return o;
}

}  // namespace eptv
