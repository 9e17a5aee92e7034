// Device helpers: principal-branch complex power for kappa(w) = 1 + c w^p.
#pragma once

#include <cuda_runtime.h>

namespace frkc2 {

// Principal square root of x + i y (branch cut on the negative real axis; the sign of a
// zero imaginary part selects the side, as in C99 csqrt).
template <class T>
__device__ __forceinline__ void csqrt_principal(T x, T y, T& rr, T& ri) {
  const T r = hypot(x, y);
  if (r == T(0)) {
    rr = T(0);
    ri = y;
    return;
  }
  if (x >= T(0)) {
    const T t = sqrt((r + x) * T(0.5));
    rr = t;
    ri = y / (T(2) * t);
  } else {
    const T t = sqrt((r - x) * T(0.5));
    rr = fabs(y) / (T(2) * t);
    ri = copysign(t, y);
  }
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
