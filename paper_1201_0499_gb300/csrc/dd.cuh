// Device double-double ("double-word") arithmetic for sm_103a.
//
// The paper's stated target precision is double double (Sections 1 and 3.2).
// A real double-double here is an unevaluated sum h + l of two doubles.  The
// operations below are built from the classic error-free transformations:
//
//   * TwoProd with a fused multiply-add (Dekker 1971; exact with an FMA):
//       p = RN(a*b),  e = fma(a, b, -p)   =>  a*b = p + e exactly.
//   * FastTwoSum (Dekker 1971): for |a| >= |b|,
//       s = RN(a+b),  e = b - (s - a)     =>  a+b = s + e exactly.
//
// On GB300 a double-precision instruction costs the FP64 pipe 16 SM cycles
// per warp (measured: about 1.8 lane-FMAs per SM per clock), while integer
// and single-precision instructions issue about 40-70 times faster.  The
// library is therefore shaped to minimise FP64 instructions:
//
//   * TwoSum of arbitrary magnitudes is FastTwoSum after ordering the two
//     operands by magnitude with integer compares and selects on the bit
//     patterns (|x| >= |y| iff (bits(x) & ~sign) >= (bits(y) & ~sign) as
//     unsigned integers, for finite x, y).  3 FP64 instructions instead of 6.
//   * A product that only feeds a sum is not renormalised (dot2: its low
//     word may be a few ulps of the high word); its rounding error is still
//     O(u^2) relative to the product of the operands' magnitudes, which is
//     the normwise error measure of the evaluation.  A product that feeds
//     another product is renormalised (dot2n, 3 more instructions): in a
//     chain of L unnormalised products the low word grows like L ulps and
//     the dropped low*low term like L^2 u^2 per step, which long chains
//     (high exponents, many variables) cannot afford.  Sums are kept
//     unnormalised and renormalised once, when they are stored.
//   * The basic product is a double-double dot product of length two,
//       z = a1*b1 + a2*b2,
//     which is one real or imaginary part of a complex product.  Cost:
//     2 DMUL + 6 DFMA + 5 DADD = 13 FP64 instructions.
//
// Every FP64 operation is written with an explicit _rn intrinsic so that the
// compiler cannot contract or reassociate what the transformations need
// separately rounded.
#pragma once

#include <cstdint>

namespace pe {

struct dd {
  double h, l;
};

// Order (a, b) by magnitude: big = the one of larger |.|.  Written in PTX so
// that the sign mask stays an integer AND: from plain C++ the compiler
// recognises the mask as fabs() and emits an FP64 instruction per operand
// (measured with the FP64 instruction counters: 5 FP64 instructions per
// TwoSum instead of 3).
__device__ __forceinline__ void order_by_magnitude(double a, double b, double &big, double &small) {
  unsigned long long hi, lo;
  asm("{\n\t"
      ".reg .pred p;\n\t"
      ".reg .b64 ma, mb;\n\t"
      "and.b64 ma, %2, 0x7fffffffffffffff;\n\t"
      "and.b64 mb, %3, 0x7fffffffffffffff;\n\t"
      "setp.gt.u64 p, mb, ma;\n\t"
      "selp.b64 %0, %3, %2, p;\n\t"
      "selp.b64 %1, %2, %3, p;\n\t"
      "}"
      : "=l"(hi), "=l"(lo)
      : "l"(__double_as_longlong(a)), "l"(__double_as_longlong(b)));
  big = __longlong_as_double(static_cast<long long>(hi));
  small = __longlong_as_double(static_cast<long long>(lo));
}

// Exact a + b = s + e for finite a, b (FastTwoSum after ordering by magnitude
// on the integer pipe).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e) {
  double big, small;
  order_by_magnitude(a, b, big, small);
  s = __dadd_rn(big, small);
  const double z = __dsub_rn(s, big);
  e = __dsub_rn(small, z);
}

// a1*b1 + a2*b2 in double-double, unnormalised result.
__device__ __forceinline__ dd dot2(dd a1, dd b1, dd a2, dd b2) {
  const double p1 = __dmul_rn(a1.h, b1.h);
  const double p2 = __dmul_rn(a2.h, b2.h);
  const double e1 = __fma_rn(a1.h, b1.h, -p1);  // a1.h*b1.h = p1 + e1 exactly
  const double e2 = __fma_rn(a2.h, b2.h, -p2);  // a2.h*b2.h = p2 + e2 exactly
  double s, es;
  two_sum(p1, p2, s, es);                       // p1 + p2 = s + es exactly
  double t = __dadd_rn(e1, e2);
  t = __fma_rn(a1.h, b1.l, t);
  t = __fma_rn(a1.l, b1.h, t);
  t = __fma_rn(a2.h, b2.l, t);
  t = __fma_rn(a2.l, b2.h, t);
  t = __dadd_rn(t, es);
  return dd{s, t};
}

// Renormalise: h = RN(h + l), l = the exact remainder (3 FP64 instructions).
__device__ __forceinline__ dd normalize(dd x) {
  double s, e;
  two_sum(x.h, x.l, s, e);
  return dd{s, e};
}

// a1*b1 + a2*b2 in double-double, renormalised (16 FP64 instructions).
__device__ __forceinline__ dd dot2n(dd a1, dd b1, dd a2, dd b2) { return normalize(dot2(a1, b1, a2, b2)); }

// acc + x, unnormalised (5 FP64 instructions).
__device__ __forceinline__ dd add(dd acc, dd x) {
  double s, es;
  two_sum(acc.h, x.h, s, es);
  double t = __dadd_rn(acc.l, x.l);
  t = __dadd_rn(t, es);
  return dd{s, t};
}

// x * k for a small integer k held exactly in a double (3 FP64 instructions).
__device__ __forceinline__ dd scale(dd x, double k) {
  const double p = __dmul_rn(x.h, k);
  const double e = __fma_rn(x.h, k, -p);
  return dd{p, __fma_rn(x.l, k, e)};
}

// Product of two double-doubles, renormalised (7 FP64 instructions).
__device__ __forceinline__ dd mul(dd a, dd b) {
  const double p = __dmul_rn(a.h, b.h);
  double t = __fma_rn(a.h, b.h, -p);
  t = __fma_rn(a.h, b.l, t);
  t = __fma_rn(a.l, b.h, t);
  return normalize(dd{p, t});
}

// 1 / d for a double-double d: the double reciprocal q of d.h refined by one
// Newton step, q + q (1 - d q), with the residual 1 - d q formed from an
// exact product (error about 2 u^2 relative).
__device__ __forceinline__ dd recip(dd d) {
  const double q = __ddiv_rn(1.0, d.h);
  const double p = __dmul_rn(d.h, q);
  const double pe = __fma_rn(d.h, q, -p);  // d.h q = p + pe exactly
  double e = __dsub_rn(1.0, p);            // exact: p is within an ulp of 1
  e = __dsub_rn(e, pe);
  e = __fma_rn(-d.l, q, e);
  return normalize(dd{q, __dmul_rn(q, e)});
}

// The double equal to an integer 1 <= a < 2^31, assembled from a's bits on
// the integer pipe (biased exponent 1023 + e for a's leading one at bit e,
// the bits below it as the fraction): a conversion instruction would take a
// slot of the FP64 pipe, the bound of the evaluation kernels.
__device__ __forceinline__ double int_as_double(int a) {
  const unsigned u = static_cast<unsigned>(a);
  const int e = 31 - __clz(u);
  const unsigned long long frac = (static_cast<unsigned long long>(u) << (52 - e)) & 0x000FFFFFFFFFFFFFULL;
  return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(1023 + e) << 52) | frac));
}

__device__ __forceinline__ dd negate_if(dd x, unsigned long long sign_mask) {
  return dd{__longlong_as_double(__double_as_longlong(x.h) ^ static_cast<long long>(sign_mask)),
            __longlong_as_double(__double_as_longlong(x.l) ^ static_cast<long long>(sign_mask))};
}

__device__ __forceinline__ double negate_if(double x, unsigned long long sign_mask) {
  return __longlong_as_double(__double_as_longlong(x) ^ static_cast<long long>(sign_mask));
}

__device__ __forceinline__ dd select(bool take_a, dd a, dd b) {
  const long long ah = __double_as_longlong(a.h), al = __double_as_longlong(a.l);
  const long long bh = __double_as_longlong(b.h), bl = __double_as_longlong(b.l);
  return dd{__longlong_as_double(take_a ? ah : bh), __longlong_as_double(take_a ? al : bl)};
}

__device__ __forceinline__ double select(bool take_a, double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  return __longlong_as_double(take_a ? ia : ib);
}

__device__ __forceinline__ dd shfl_xor(dd x, int m) {
  return dd{__shfl_xor_sync(0xffffffffu, x.h, m), __shfl_xor_sync(0xffffffffu, x.l, m)};
}

__device__ __forceinline__ double shfl_xor(double x, int m) { return __shfl_xor_sync(0xffffffffu, x, m); }

}  // namespace pe
