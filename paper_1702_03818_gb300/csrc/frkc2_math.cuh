// Device helpers: principal-branch complex power for kappa(w) = 1 + c w^p.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

namespace frkc2 {

// Principal square root of x + i y (branch cut on the negative real axis; the sign of a
// zero imaginary part selects the side, as in C99 csqrt), from the half-angle formulas
//   t = sqrt((|w| + |x|) / 2),  sqrt(w) = (t, y / (2t)) for x >= 0, (|y| / (2t), sign(y) t) else,
// with both square roots and the division taken from two reciprocal square roots:
// |w| = m rsqrt(m), m = x^2 + y^2, and with q = rsqrt((|w| + |x|)/2): t = ((|w| + |x|)/2) q,
// |y| / (2t) = |y| q / 2.  On GB300's narrow FP64 pipe this is about half the cost of hypot,
// sqrt and a division.  (m is formed without rescaling: |w| below ~1e-154 or above ~1e154
// in FP64 (1e-19 / 1e19 in FP32) loses accuracy, far outside the states of a diffusion run.)
// Reciprocal square root: CUDA's rsqrt in FP64; in FP32 the hardware approximation with
// subnormal inputs flushed to zero (rsqrt.approx.ftz: the same accuracy for normal inputs,
// without the subnormal handling; csqrt_principal keeps its inputs normal).
__device__ __forceinline__ double rsqrt_n(double a) { return rsqrt(a); }
__device__ __forceinline__ float rsqrt_n(float a) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
  return r;
}

template <class T>
__device__ __forceinline__ void csqrt_principal(T x, T y, T& rr, T& ri) {
  const T m = x * x + y * y;
  // w = 0, or in FP32 a modulus below ~1e-19 (m subnormal, which rsqrt.approx.ftz would take
  // as zero): sqrt(w) taken as (0, y)
  if (m == T(0) || (std::is_same<T, float>::value && m < T(1.17549435e-38f))) {
    rr = T(0);
    ri = y;
    return;
  }
  const T r = m * rsqrt_n(m);
  const T a = (r + fabs(x)) * T(0.5);
  const T q = rsqrt_n(a);
  const T t = a * q;
  const T h = T(0.5) * fabs(y) * q;
  if (x >= T(0)) {
    rr = t;
    ri = copysign(h, y);
  } else {
    rr = h;
    ri = copysign(t, y);
  }
}

// kappa(w) = 1 + c w^2.5 = 1 + c w^2 sqrt(w) for complex w = u + i v (principal branch).
template <class T>
__device__ __forceinline__ void kappa_power25(T u, T v, T c, T& kr, T& ki) {
  T sr, si;
  csqrt_principal<T>(u, v, sr, si);  // sqrt(0) = 0, so 0^2.5 = 0 needs no test
  const T qr = u * u - v * v, qi = T(2) * u * v;
  kr = T(1) + c * (qr * sr - qi * si);
  ki = c * (qr * si + qi * sr);
}

// kappa(w) = 1 + c w^p for complex w = u + i v on the principal branch, 0^p = 0 (p > 0).
// p = 2.5 uses w^2 * sqrt(w); other exponents use the polar form |w|^p e^{i p arg w}.
template <class T>
__device__ __forceinline__ void kappa_power(T u, T v, T c, T p, T& kr, T& ki) {
  T wr = T(0), wi = T(0);
  if (u != T(0) || v != T(0)) {
    if (p == T(2.5)) {
      T sr, si;
      csqrt_principal<T>(u, v, sr, si);
      const T qr = u * u - v * v, qi = T(2) * u * v;
      wr = qr * sr - qi * si;
      wi = qr * si + qi * sr;
    } else {
      const T r = hypot(u, v), th = atan2(v, u);
      const T rp = pow(r, p);
      T sn, cs;
      sincos(p * th, &sn, &cs);
      wr = rp * cs;
      wi = rp * sn;
    }
  }
  kr = T(1) + c * wr;
  ki = c * wi;
}

}  // namespace frkc2
