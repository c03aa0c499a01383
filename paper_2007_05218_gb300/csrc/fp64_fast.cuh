// FP64 helpers that keep work off GB300's narrow FP64 pipe.
//
// Reciprocal, reciprocal square root and square root: a hardware
// approximation (PTX rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64, executed by
// the special-function unit, not the FP64 pipe) refined by one third-order
// Newton-Raphson step (Householder's method of order 3) in fused multiply-adds:
//   1/x:       e = 1 - x y,    y <- y (1 + e + e^2)
//   1/sqrt(x): e = 1 - x y^2,  y <- y (1 + e/2 + 3 e^2 / 8)
// A seed with relative error eps leaves O(eps^3) plus a few roundings: the
// results are within a few ulp, for 3 to 6 FP64-pipe instructions instead of
// the ~10 pipe slots an IEEE divide or square root takes.  Arguments must be
// non-zero normal numbers (positive for the square roots): the callers pass
// densities, pressures, sound-speed products and wave-speed differences that
// the method keeps away from zero.
//
// Sign tests and min/max on the bit patterns run on the integer pipe and give
// the same answers as the FP64 comparisons for every finite non-NaN input
// (products that underflow to zero aside).
#pragma once

namespace hydro {

__device__ __forceinline__ double nr_rcp(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x, y, 1.0);
  return fma(y, fma(e, e, e), y);
}

__device__ __forceinline__ double nr_rsqrt(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-x * y, y, 1.0);
  return fma(y * e, fma(e, 0.375, 0.5), y);
}

__device__ __forceinline__ double nr_sqrt(double x) { return x * nr_rsqrt(x); }

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }

// x > 0
__device__ __forceinline__ bool is_pos(double x) { return dbits(x) > 0; }
// x < 0 (-0.0 is not negative)
__device__ __forceinline__ bool is_neg(double x) {
  const long long b = dbits(x);
  return b < 0 && (b << 1) != 0;
}
// x >= 0
__device__ __forceinline__ bool is_nonneg(double x) { return !is_neg(x); }
// x * y > 0: same sign and neither is zero
__device__ __forceinline__ bool same_sign(double x, double y) {
  const long long a = dbits(x), b = dbits(y);
  return (a ^ b) >= 0 && (a << 1) != 0 && (b << 1) != 0;
}
// integer key that orders like the double (negatives flipped below positives)
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dmin(double a, double b) { return dkey(a) <= dkey(b) ? a : b; }
__device__ __forceinline__ double dmax(double a, double b) { return dkey(a) >= dkey(b) ? a : b; }
// a > b
__device__ __forceinline__ bool dgt(double a, double b) { return dkey(a) > dkey(b); }

}  // namespace hydro
