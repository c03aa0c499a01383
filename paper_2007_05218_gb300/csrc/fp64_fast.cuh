// Arithmetic helpers for the stage kernels, for both compute types.
//
// FP64 (double): GB300's FP64 pipe is narrow, so reciprocal, reciprocal square
// root and square root use a hardware approximation (PTX rcp.approx.ftz.f64 /
// rsqrt.approx.ftz.f64, executed by the special-function unit, not the FP64
// pipe) refined by one third-order Newton-Raphson step (Householder's method
// of order 3) in fused multiply-adds:
//   1/x:       e = 1 - x y,    y <- y (1 + e + e^2)
//   1/sqrt(x): e = 1 - x y^2,  y <- y (1 + e/2 + 3 e^2 / 8)
// A seed with relative error eps (about 2^-20 here) leaves O(eps^3) plus a few
// roundings: measured on GB300 over normal arguments from 2^-1000 to 2^1000
// (tests/fp64_helpers_check.cu), the reciprocal is within 1.0 ulp of the
// correctly rounded one, the square root (x times its reciprocal square root)
// within 1.7 ulp and the reciprocal square root within 1.25 x 2^-53 relative,
// for 3 to 6 FP64-pipe instructions instead of the ~10 pipe slots an IEEE
// divide or square root takes.  Arguments must be non-zero normal numbers (positive for the square
// roots): the callers pass densities, pressures, sound-speed products and
// wave-speed differences that the method keeps away from zero.
//
// FP32 (float, mixed precision): the CUDA single-precision reciprocal and
// square root (correctly rounded) and rsqrtf (within 2 ulp).
//
// FP64 sign tests, min/max, halvings and the |x| > 2|y| test work on the bit
// patterns, in their two 32-bit halves (64-bit integer operations on the
// patterns were measured to cost FP64-pipe time), and give the same answers as
// floating-point operations for every finite non-NaN input (products that
// underflow to zero aside).  FP32 uses the native instructions.  The generic
// templates state the semantics.
#pragma once

namespace hydro {

// FP64 product on the integer pipe.  GB300's FP64 pipe is the scarce unit of
// the FP64 kernels while its integer pipe idles, and a correctly rounded
// product needs only 32-bit integer work: the 106-bit product of the two
// 53-bit significands from four 32 x 32 -> 64-bit multiply-adds, a one-bit
// normalisation, round to nearest even on the dropped bits (guard bit, then
// sticky or the kept lsb), and the exponent added to the significand with its
// leading bit (so that a carry out of the rounding raises the exponent, and
// rounding past the largest binade gives infinity).  Bitwise __dmul_rn for
// normal or zero operands whose product is normal or zero; for any other
// operands (subnormal, infinite or NaN, or a product that underflows or
// overflows) it sets `bad`, and the caller recomputes with the FP64
// instruction.  tests/fp64_helpers_check.cu compares it with __dmul_rn bit
// for bit over every exponent pair.
__device__ __forceinline__ double imul_rn(double a, double b, unsigned& bad) {
  const unsigned ah = (unsigned)__double2hiint(a), al = (unsigned)__double2loint(a);
  const unsigned bh = (unsigned)__double2hiint(b), bl = (unsigned)__double2loint(b);
  // exponent fields in place (bits 20..30 of the high words)
  const unsigned xa = ah & 0x7ff00000u, xb = bh & 0x7ff00000u;
  const unsigned mah = (ah & 0xfffffu) | 0x100000u, mbh = (bh & 0xfffffu) | 0x100000u;
  // P = ma mb = up 2^64 + w1 2^32 + w0, up < 2^42
  const unsigned long long ll = (unsigned long long)al * bl;
  const unsigned long long t1 = (unsigned long long)mah * bl + (ll >> 32);
  const unsigned long long t2 = (unsigned long long)al * mbh + (unsigned)t1;
  const unsigned w0 = (unsigned)ll, w1 = (unsigned)t2;
  const unsigned long long up = (unsigned long long)mah * mbh + ((t1 >> 32) + (t2 >> 32));
  const unsigned uh = (unsigned)(up >> 32), ul = (unsigned)up;
  const unsigned top = (uh >> 9) & 1u;  // P >= 2^105
  const unsigned sh = 12u - top;        // the 53 kept bits end at bit 52 + top of P
  const unsigned ml = __funnelshift_l(w1, ul, sh), mh = __funnelshift_l(ul, uh, sh);
  // round to nearest even: the dropped bits of w1 (guard bit first; their low
  // sh >= 11 bits are zero, so the lowest one can carry the sticky bit of w0)
  // plus 2^31 - 1 + lsb carry out of 32 bits exactly when the kept part rounds up
  const unsigned rem = (w1 << sh) | min(w0, 1u);
  const unsigned inc = (unsigned)(((unsigned long long)rem + 0x7fffffffu + (ml & 1u)) >> 32);
  const unsigned long long m = (((unsigned long long)mh << 32) | ml) + inc;
  // result high word: exponent field (xa + xb + top - 1023, in place) plus the
  // significand with its leading bit, which adds the one the field lacks
  const unsigned ex = xa + xb + (top << 20) - (1024u << 20);  // (biased exponent - 1) << 20, mod 2^32
  const unsigned sign = (ah ^ bh) & 0x80000000u;
  const bool za = ((ah & 0x7fffffffu) | al) == 0u, zb = ((bh & 0x7fffffffu) | bl) == 0u;
  const bool zero = (za & (xb != 0x7ff00000u)) | (zb & (xa != 0x7ff00000u));  // zero times a finite number
  // normal operands (field 1..2046) and a normal product (biased exponent 1..2046 before rounding)
  const bool ok = ((xa - 0x100000u < 0x7fe00000u) & (xb - 0x100000u < 0x7fe00000u) & (ex < 0x7fe00000u)) | zero;
  bad |= ok ? 0u : 1u;
  return zero ? __hiloint2double((int)sign, 0)
              : __hiloint2double((int)((ex + (unsigned)(m >> 32)) | sign), (int)(unsigned)m);
}

// The FP64 multiply instruction where the integer product set `bad`: volatile,
// so that the compiler keeps it inside the rarely taken recomputation instead
// of issuing it in every warp.
__device__ __forceinline__ double dmul_insn(double a, double b) {
  double r;
  asm volatile("mul.rn.f64 %0, %1, %2;" : "=d"(r) : "d"(a), "d"(b));
  return r;
}

// Multiplication policies for the stage arithmetic that is written once for
// both forms: IntMul forms FP64 products on the integer pipe and records in
// `bad` whether any could not be formed there; InsnMul uses the FP64
// instruction (the recomputation of a lane that IntMul flagged).  Both are
// bitwise __dmul_rn, and FP32 products are plain in both.  Used where the
// product is an operand of something other than an addition, so that no fused
// multiply-add is split.
struct IntMul {
  unsigned bad = 0u;
  __device__ __forceinline__ double operator()(double a, double b) { return imul_rn(a, b, bad); }
  __device__ __forceinline__ float operator()(float a, float b) { return a * b; }
};
struct InsnMul {
  __device__ __forceinline__ double operator()(double a, double b) { return dmul_insn(a, b); }
  __device__ __forceinline__ float operator()(float a, float b) { return a * b; }
};
// The FP64 multiply without the integer pipe (the persistent kernel's stage
// bodies, where the integer-pipe products were measured slower): the same
// bits as IntMul, so that both forms of a step agree bit for bit.
struct PlainMul {
  __device__ __forceinline__ double operator()(double a, double b) { return __dmul_rn(a, b); }
  __device__ __forceinline__ float operator()(float a, float b) { return a * b; }
};

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

// The same with the two products (and the square root's third) taken by a
// multiplication policy.
template <typename M>
__device__ __forceinline__ double nr_rsqrt(double x, M& mul) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  const double e = fma(-mul(x, y), y, 1.0);
  return fma(mul(y, e), fma(e, 0.375, 0.5), y);
}
template <typename M>
__device__ __forceinline__ double nr_sqrt(double x, M& mul) { return mul(x, nr_rsqrt(x, mul)); }

__device__ __forceinline__ float nr_rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ float nr_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ float nr_sqrt(float x) { return sqrtf(x); }
template <typename M>
__device__ __forceinline__ float nr_rsqrt(float x, M&) { return rsqrtf(x); }
template <typename M>
__device__ __forceinline__ float nr_sqrt(float x, M&) { return sqrtf(x); }

// bit patterns as signed integers of the same width
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ int dbits(float x) { return __float_as_int(x); }
__device__ __forceinline__ double from_bits(long long b) { return __longlong_as_double(b); }
__device__ __forceinline__ float from_bits(int b) { return __int_as_float(b); }

// x > 0
template <typename R>
__device__ __forceinline__ bool is_pos(R x) { return dbits(x) > 0; }
// x < 0 (-0.0 is not negative)
template <typename R>
__device__ __forceinline__ bool is_neg(R x) {
  const auto b = dbits(x);
  return b < 0 && (b << 1) != 0;
}
// x >= 0
template <typename R>
__device__ __forceinline__ bool is_nonneg(R x) { return !is_neg(x); }
// x * y > 0: same sign and neither is zero
template <typename R>
__device__ __forceinline__ bool same_sign(R x, R y) {
  const auto a = dbits(x), b = dbits(y);
  return (a ^ b) >= 0 && (a << 1) != 0 && (b << 1) != 0;
}
// x * y < 0: opposite signs and neither is zero
template <typename R>
__device__ __forceinline__ bool opp_sign(R x, R y) {
  const auto a = dbits(x), b = dbits(y);
  return (a ^ b) < 0 && (a << 1) != 0 && (b << 1) != 0;
}
// integer key that orders like the value (negatives flipped below positives)
__device__ __forceinline__ long long dkey(double x) {
  const long long b = dbits(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ int dkey(float x) {
  const int b = dbits(x);
  return b ^ ((b >> 31) & 0x7fffffff);
}
template <typename R>
__device__ __forceinline__ R dmin(R a, R b) { return dkey(a) <= dkey(b) ? a : b; }
template <typename R>
__device__ __forceinline__ R dmax(R a, R b) { return dkey(a) >= dkey(b) ? a : b; }
// a > b
template <typename R>
__device__ __forceinline__ bool dgt(R a, R b) { return dkey(a) > dkey(b); }
// x / 2, correctly rounded
template <typename R>
__device__ __forceinline__ R half_of(R x) { return R(0.5) * x; }
// 2 x, correctly rounded
template <typename R>
__device__ __forceinline__ R twice_of(R x) { return R(2) * x; }
// |x| > 2 |y|
template <typename R>
__device__ __forceinline__ bool abs_gt_twice(R x, R y) { return fabs(x) > R(2) * fabs(y); }

// FP64 forms on the two 32-bit halves of each double (sign, exponent and top
// mantissa bits in the high word): 64-bit integer operations on the bit
// patterns were measured to cost FP64-pipe time on GB300, 32-bit ones run on
// the integer pipe.  Same results as the generic forms (the ordering key
// flips the magnitude bits of negative numbers; -0.0 orders below +0.0).
// They combine their tests with bitwise operators and select rather than
// branch: a data-dependent branch that splits a warp makes the FP64
// instructions after it issue once per side until the warp reconverges.
__device__ __forceinline__ bool hw_nz(int hi, unsigned lo) { return ((hi & 0x7fffffff) | (int)lo) != 0; }
template <>
__device__ __forceinline__ bool is_pos<double>(double x) {
  const int h = __double2hiint(x);
  return (h > 0) | ((h == 0) & (__double2loint(x) != 0));
}
template <>
__device__ __forceinline__ bool is_neg<double>(double x) {
  const int h = __double2hiint(x);
  return (h < 0) & hw_nz(h, (unsigned)__double2loint(x));
}
template <>
__device__ __forceinline__ bool same_sign<double>(double x, double y) {
  const int hx = __double2hiint(x), hy = __double2hiint(y);
  return ((hx ^ hy) >= 0) & hw_nz(hx, (unsigned)__double2loint(x)) & hw_nz(hy, (unsigned)__double2loint(y));
}
template <>
__device__ __forceinline__ bool opp_sign<double>(double x, double y) {
  const int hx = __double2hiint(x), hy = __double2hiint(y);
  return ((hx ^ hy) < 0) & hw_nz(hx, (unsigned)__double2loint(x)) & hw_nz(hy, (unsigned)__double2loint(y));
}
template <>
__device__ __forceinline__ bool dgt<double>(double a, double b) {
  const int ha = __double2hiint(a), hb = __double2hiint(b);
  const int sa = ha >> 31, sb = hb >> 31;  // all ones for negative numbers
  const int ka = ha ^ (sa & 0x7fffffff), kb = hb ^ (sb & 0x7fffffff);
  const unsigned ja = (unsigned)__double2loint(a) ^ (unsigned)sa, jb = (unsigned)__double2loint(b) ^ (unsigned)sb;
  return (ka > kb) | ((ka == kb) & (ja > jb));
}
template <>
__device__ __forceinline__ double dmin<double>(double a, double b) { return dgt(a, b) ? b : a; }
template <>
__device__ __forceinline__ double dmax<double>(double a, double b) { return dgt(b, a) ? b : a; }
// x > 0 and not NaN (+inf included), on the bit pattern: 0 < bits <= that of +inf
__device__ __forceinline__ bool pos_not_nan(double x) {
  const int h = __double2hiint(x);
  const unsigned l = (unsigned)__double2loint(x);
  return ((h > 0) | ((h == 0) & (l != 0u))) & ((h < 0x7ff00000) | ((h == 0x7ff00000) & (l == 0u)));
}
// x / 2 without an FP64 instruction.  For 2^-1021 <= |x| < inf it is an
// exponent decrement of the high word.  Below that range the magnitude bits
// (exponent field 0 or 1) read as an integer M give |x| = M 2^-1074, so x / 2
// is the pattern M / 2 rounded half to even; zero stays zero.  Infinities and
// NaN are returned unchanged.
template <>
__device__ __forceinline__ double half_of<double>(double x) {
  const int hi = __double2hiint(x);
  const unsigned lo = (unsigned)__double2loint(x);
  const unsigned mh = (unsigned)hi & 0x7fffffffu;
  constexpr unsigned E2 = 2u << 20, INF = 0x7ff00000u;
  const bool dec = mh - E2 < INF - E2, keep = mh >= INF;
  const unsigned ql = (lo >> 1) | (mh << 31), qh = mh >> 1;
  const unsigned rl = ql + (lo & ql & 1u);  // a dropped half rounds an odd result up
  const unsigned rh = (qh + (rl < ql ? 1u : 0u)) | ((unsigned)hi & 0x80000000u);
  const unsigned oh = dec ? (unsigned)hi - (1u << 20) : keep ? (unsigned)hi : rh;
  return __hiloint2double((int)oh, (int)(dec | keep ? lo : rl));
}
// 2 x without an FP64 instruction: an exponent increment of the high word for
// 2^-1022 <= |x| < 2^1023, the magnitude pattern doubled for |x| below that
// (exact, also where it becomes normal), infinity of x's sign for
// 2^1023 <= |x| < inf; infinities and NaN are returned unchanged.
template <>
__device__ __forceinline__ double twice_of<double>(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mh = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  const bool sub = mh < 0x00100000u, big = mh >= 0x7fe00000u, special = mh >= 0x7ff00000u;
  unsigned rh = hi + 0x00100000u, rl = lo;
  if (sub) {
    rh = ((mh << 1) | (lo >> 31)) | sign;
    rl = lo << 1;
  }
  if (big) {
    rh = special ? hi : (sign | 0x7ff00000u);
    rl = special ? lo : 0u;
  }
  return __hiloint2double((int)rh, (int)rl);
}
// |x| > 2 |y| for finite x, y, on the magnitude bits: 2|y| is an exponent
// increment of a normal |y| and the magnitude pattern doubled for a
// subnormal one (which is exact, also where it becomes normal); a normal |y|
// of 2^1023 or more makes 2|y| overflow, which no finite |x| exceeds.
template <>
__device__ __forceinline__ bool abs_gt_twice<double>(double x, double y) {
  const unsigned hx = (unsigned)__double2hiint(x) & 0x7fffffffu, lx = (unsigned)__double2loint(x);
  const unsigned hy = (unsigned)__double2hiint(y) & 0x7fffffffu, ly = (unsigned)__double2loint(y);
  const bool nrm = hy >= (1u << 20);
  const unsigned h2 = nrm ? hy + (1u << 20) : (hy << 1) | (ly >> 31);
  const unsigned l2 = nrm ? ly : ly << 1;
  return (hy < 0x7fe00000u) & ((hx > h2) | ((hx == h2) & (lx > l2)));
}

// FP64 -> FP32 rounded to nearest even, on the integer pipe (the conversion
// instruction occupies the FP64 pipe), as a bit pattern.  Exact for results
// in the normal FP32 range (|x| in [2^-126, 2^128), where a carry out of the
// mantissa raises the exponent and rounds the largest values to infinity)
// and for |x| < 2^-150 (zero, of x's sign).  Everything else (results that
// are FP32 subnormals, |x| >= 2^128, infinities, NaN) sets `rare`, and the
// caller converts those with the instruction.
__device__ __forceinline__ unsigned narrow_bits(double x, bool& rare) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned mh = hi & 0x7fffffffu, sign = hi & 0x80000000u;
  // exponent field e = mh >> 20: a normal FP32 result for 897 <= e <= 1150
  const bool normal = mh - (897u << 20) < ((1151u - 897u) << 20);
  const bool tiny = mh < (873u << 20);  // |x| < 2^-150
  const unsigned m = ((mh - (896u << 20)) << 3) | (lo >> 29);
  const unsigned rem = lo & 0x1fffffffu;
  const unsigned up = (rem > 0x10000000u) | ((rem == 0x10000000u) & (m & 1u));
  rare = !normal & !tiny;
  return tiny ? sign : sign | (m + up);
}

// FP32 keeps its comparisons and min/max native: the FP32 units are not the
// scarce resource there, and one native instruction replaces the several
// integer ones of the bit-pattern forms (same results for finite inputs).
template <>
__device__ __forceinline__ float dmin<float>(float a, float b) { return fminf(a, b); }
template <>
__device__ __forceinline__ float dmax<float>(float a, float b) { return fmaxf(a, b); }
template <>
__device__ __forceinline__ bool dgt<float>(float a, float b) { return a > b; }
template <>
__device__ __forceinline__ bool is_pos<float>(float x) { return x > 0.0f; }
template <>
__device__ __forceinline__ bool is_neg<float>(float x) { return x < 0.0f; }
template <>
__device__ __forceinline__ bool same_sign<float>(float x, float y) { return x * y > 0.0f; }
template <>
__device__ __forceinline__ bool opp_sign<float>(float x, float y) { return x * y < 0.0f; }

}  // namespace hydro
