// Complex block floating point with 128-bit mantissas, on the integer pipes.
//
// Why: on GB300 a double-precision instruction issues at about 1.8 lanes per
// SM per clock, a 32-bit integer multiply-add, shift or carry-add at about 64
// (measured).  Extended precision built from 32-bit integer limbs therefore
// costs far less time than double-double built from FP64 operations, and it is
// more precise.
//
// Format.  A complex number is (A + iB) * 2^e with A and B held in
// sign-magnitude form: a 128-bit magnitude in four 32-bit limbs (limb 0 least
// significant) and a sign bit each, and one shared 32-bit exponent e.  Values
// that feed further products are normalised: max(|A|, |B|) in [2^125, 2^126)
// (one bit of headroom for sums); zero is all-zero magnitudes with
// e = kZeroExp.  Rounding is truncation; every product keeps the top 128 bits
// of the 256-bit product of the magnitudes (the three lowest columns of
// partial products are dropped), so each operation errs by a few units in the
// 2^-125 place relative to the product of the operands' magnitudes --
// normwise, which is the error measure of the evaluation -- about 2^-120
// after renormalisation.
//
// Lane pairs (as in the double-double kernel): lanes 2q and 2q+1 hold the
// real and the imaginary part of the values of point q.  A lane holds one
// magnitude and sign; both lanes of a pair hold the same exponent.
#pragma once

#include <cstdint>

#include "dd.cuh"

namespace pe {
namespace wide {

constexpr int32_t kZeroExp = -(1 << 28);
constexpr uint32_t kSignBit = 0x80000000u;

struct Mag {
  uint32_t w0, w1, w2, w3;
};

// One component held by a lane: magnitude, sign (0 or kSignBit), exponent.
struct WV {
  Mag m;
  uint32_t s;
  int32_t e;
};

// A full complex value (both components), as stored in memory: 12 words,
// re limbs, im limbs, signs (bit 31 re, bit 30 im), exponent, 2 spare.
struct WF {
  Mag re, im;
  uint32_t signs;
  int32_t e;
};

__device__ __forceinline__ WF load_wf(const uint32_t *p) {
  const uint4 a = __ldg(reinterpret_cast<const uint4 *>(p));
  const uint4 b = __ldg(reinterpret_cast<const uint4 *>(p) + 1);
  const uint2 c = __ldg(reinterpret_cast<const uint2 *>(p + 8));
  return WF{Mag{a.x, a.y, a.z, a.w}, Mag{b.x, b.y, b.z, b.w}, c.x, static_cast<int32_t>(c.y)};
}

__device__ __forceinline__ WF load_wf_coherent(const uint32_t *p) {
  const uint4 a = reinterpret_cast<const uint4 *>(p)[0];
  const uint4 b = reinterpret_cast<const uint4 *>(p)[1];
  const uint2 c = *reinterpret_cast<const uint2 *>(p + 8);
  return WF{Mag{a.x, a.y, a.z, a.w}, Mag{b.x, b.y, b.z, b.w}, c.x, static_cast<int32_t>(c.y)};
}

__device__ __forceinline__ void store_wf(uint32_t *p, const WF &v) {
  reinterpret_cast<uint4 *>(p)[0] = make_uint4(v.re.w0, v.re.w1, v.re.w2, v.re.w3);
  reinterpret_cast<uint4 *>(p)[1] = make_uint4(v.im.w0, v.im.w1, v.im.w2, v.im.w3);
  reinterpret_cast<uint4 *>(p)[2] = make_uint4(v.signs, static_cast<uint32_t>(v.e), 0u, 0u);
}

// The component c (0 real, 1 imaginary) of a full value, as a lane value.
__device__ __forceinline__ WV component(const WF &x, int c) {
  const bool re = c == 0;
  return WV{Mag{re ? x.re.w0 : x.im.w0, re ? x.re.w1 : x.im.w1, re ? x.re.w2 : x.im.w2, re ? x.re.w3 : x.im.w3},
            (re ? x.signs : (x.signs << 1)) & kSignBit, x.e};
}

__device__ __forceinline__ bool is_zero(const Mag &a) { return (a.w0 | a.w1 | a.w2 | a.w3) == 0u; }

// Top 128 bits of the 256-bit product a*b.  Columns 0..2 of the partial
// products are dropped and column 3 contributes only its high words, so the
// result is low by at most 7 units in its last place.
__device__ __forceinline__ Mag mul_hi(const Mag &a, const Mag &b) {
  uint32_t c1, c2, c3, c4;
  asm("{\n\t"
      // column 3, high words: hi(a0b3) + hi(a1b2) + hi(a2b1) + hi(a3b0) into (c1, c2)
      "mul.hi.u32      %0, %4, %11;\n\t"
      "mad.hi.cc.u32   %0, %5, %10, %0;\n\t"
      "addc.u32        %1, 0, 0;\n\t"
      "mad.hi.cc.u32   %0, %6, %9, %0;\n\t"
      "addc.u32        %1, %1, 0;\n\t"
      "mad.hi.cc.u32   %0, %7, %8, %0;\n\t"
      "addc.u32        %1, %1, 0;\n\t"
      // column 4: a1b3 + a2b2 + a3b1 into (c1, c2, c3)
      "mad.lo.cc.u32   %0, %5, %11, %0;\n\t"
      "madc.hi.cc.u32  %1, %5, %11, %1;\n\t"
      "addc.u32        %2, 0, 0;\n\t"
      "mad.lo.cc.u32   %0, %6, %10, %0;\n\t"
      "madc.hi.cc.u32  %1, %6, %10, %1;\n\t"
      "addc.u32        %2, %2, 0;\n\t"
      "mad.lo.cc.u32   %0, %7, %9, %0;\n\t"
      "madc.hi.cc.u32  %1, %7, %9, %1;\n\t"
      "addc.u32        %2, %2, 0;\n\t"
      // column 5: a2b3 + a3b2 into (c2, c3, c4)
      "mad.lo.cc.u32   %1, %6, %11, %1;\n\t"
      "madc.hi.cc.u32  %2, %6, %11, %2;\n\t"
      "addc.u32        %3, 0, 0;\n\t"
      "mad.lo.cc.u32   %1, %7, %10, %1;\n\t"
      "madc.hi.cc.u32  %2, %7, %10, %2;\n\t"
      "addc.u32        %3, %3, 0;\n\t"
      // column 6: a3b3 into (c3, c4)
      "mad.lo.cc.u32   %2, %7, %11, %2;\n\t"
      "madc.hi.u32     %3, %7, %11, %3;\n\t"
      "}"
      : "=&r"(c1), "=&r"(c2), "=&r"(c3), "=&r"(c4)
      : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(a.w3), "r"(b.w0), "r"(b.w1), "r"(b.w2), "r"(b.w3));
  return Mag{c1, c2, c3, c4};
}

// (p1 with sign s1) + (p2 with sign s2), both magnitudes < 2^126: magnitude
// and sign of the sum.
__device__ __forceinline__ Mag signed_add(const Mag &p1, uint32_t s1, const Mag &p2, uint32_t s2, uint32_t &s) {
  const uint32_t m = static_cast<uint32_t>(static_cast<int32_t>(s1 ^ s2) >> 31);  // all ones: subtract
  uint32_t r0, r1, r2, r3, cout;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "and.b32         t, %13, 1;\n\t"
      "add.cc.u32      t, t, 0xffffffff;\n\t"  // carry-in = 1 when subtracting
      "xor.b32         %4, %9, %13;\n\t"
      "addc.cc.u32     %0, %5, %4;\n\t"
      "xor.b32         %4, %10, %13;\n\t"
      "addc.cc.u32     %1, %6, %4;\n\t"
      "xor.b32         %4, %11, %13;\n\t"
      "addc.cc.u32     %2, %7, %4;\n\t"
      "xor.b32         %4, %12, %13;\n\t"
      "addc.cc.u32     %3, %8, %4;\n\t"
      "addc.u32        %4, 0, 0;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3), "=&r"(cout)
      : "r"(p1.w0), "r"(p1.w1), "r"(p1.w2), "r"(p1.w3), "r"(p2.w0), "r"(p2.w1), "r"(p2.w2), "r"(p2.w3), "r"(m));
  // subtracting and no carry out: p2 > p1, negate the difference
  const uint32_t nm = m & (cout - 1u);
  uint32_t q0, q1, q2, q3;
  asm("{\n\t"
      ".reg .u32 u;\n\t"
      "and.b32         u, %8, 1;\n\t"
      "add.cc.u32      u, u, 0xffffffff;\n\t"
      "xor.b32         %0, %4, %8;\n\t"
      "addc.cc.u32     %0, %0, 0;\n\t"
      "xor.b32         %1, %5, %8;\n\t"
      "addc.cc.u32     %1, %1, 0;\n\t"
      "xor.b32         %2, %6, %8;\n\t"
      "addc.cc.u32     %2, %2, 0;\n\t"
      "xor.b32         %3, %7, %8;\n\t"
      "addc.u32        %3, %3, 0;\n\t"
      "}"
      : "=&r"(q0), "=&r"(q1), "=&r"(q2), "=&r"(q3)
      : "r"(r0), "r"(r1), "r"(r2), "r"(r3), "r"(nm));
  s = nm ? s2 : s1;
  return Mag{q0, q1, q2, q3};
}

// Leading zeros of a 128-bit magnitude (128 for zero).
__device__ __forceinline__ int clz128(const Mag &a) {
  const int z3 = __clz(static_cast<int>(a.w3)), z2 = __clz(static_cast<int>(a.w2));
  const int z1 = __clz(static_cast<int>(a.w1)), z0 = __clz(static_cast<int>(a.w0));
  return a.w3 ? z3 : a.w2 ? 32 + z2 : a.w1 ? 64 + z1 : 96 + z0;
}

// Left shift by 0 <= n < 128.
__device__ __forceinline__ Mag shl(const Mag &a, int n) {
  Mag x = a;
  if (n >= 64) {
    x = Mag{0u, 0u, x.w0, x.w1};
    n -= 64;
  }
  if (n >= 32) {
    x = Mag{0u, x.w0, x.w1, x.w2};
    n -= 32;
  }
  return Mag{x.w0 << n, __funnelshift_l(x.w0, x.w1, n), __funnelshift_l(x.w1, x.w2, n),
             __funnelshift_l(x.w2, x.w3, n)};
}

// Right shift by n >= 0 (n >= 128 gives zero).
__device__ __forceinline__ Mag shr(const Mag &a, int n) {
  if (n >= 128) return Mag{0u, 0u, 0u, 0u};
  Mag x = a;
  if (n >= 64) {
    x = Mag{x.w2, x.w3, 0u, 0u};
    n -= 64;
  }
  if (n >= 32) {
    x = Mag{x.w1, x.w2, x.w3, 0u};
    n -= 32;
  }
  return Mag{__funnelshift_r(x.w0, x.w1, n), __funnelshift_r(x.w1, x.w2, n), __funnelshift_r(x.w2, x.w3, n),
             x.w3 >> n};
}

__device__ __forceinline__ Mag shfl_xor_mag(const Mag &a, int m) {
  return Mag{__shfl_xor_sync(0xffffffffu, a.w0, m), __shfl_xor_sync(0xffffffffu, a.w1, m),
             __shfl_xor_sync(0xffffffffu, a.w2, m), __shfl_xor_sync(0xffffffffu, a.w3, m)};
}

// Normalise a lane-pair value: the larger magnitude of the pair to
// [2^125, 2^126), both lanes shifted alike; zero pairs get kZeroExp.
__device__ __forceinline__ WV normalize_pair(const WV &v) {
  // usual case: both leading bits in the top limb, a left shift below 32
  const int lz3 = __clz(static_cast<int>(v.m.w3));
  const int lz3p = __shfl_xor_sync(0xffffffffu, lz3, 1);
  const int z3 = min(lz3, lz3p);
  if (__all_sync(0xffffffffu, z3 >= 2 && z3 < 32)) {
    const int sh = z3 - 2;
    return WV{Mag{v.m.w0 << sh, __funnelshift_l(v.m.w0, v.m.w1, sh), __funnelshift_l(v.m.w1, v.m.w2, sh),
                  __funnelshift_l(v.m.w2, v.m.w3, sh)},
              v.s, v.e - sh};
  }
  const int lz = clz128(v.m);
  const int lzp = __shfl_xor_sync(0xffffffffu, lz, 1);
  const int z = min(lz, lzp);
  if (z == 128) return WV{Mag{0u, 0u, 0u, 0u}, 0u, kZeroExp};
  const int sh = z - 2;  // leading bit to position 125
  if (sh >= 0) return WV{shl(v.m, sh), v.s, v.e - sh};
  return WV{shr(v.m, -sh), v.s, v.e - sh};
}

// y (split over the pair) times X (full value on both lanes), normalised
// when Norm:
//   re: X.re y.re - X.im y.im      im: X.re y.im + X.im y.re
// Unnormalised, the pair's larger magnitude lies in [2^121, 2^125) (the
// product of normalised operands, top half, plus one sum); a product of such
// an operand keeps 2 fewer significant bits, still about 2^-118, so chains
// normalise only every second product.
template <bool Norm = true>
__device__ __forceinline__ WV mul_x(const WV &y, const WF &X, int c) {
  const Mag yp = shfl_xor_mag(y.m, 1);
  const uint32_t sp = __shfl_xor_sync(0xffffffffu, y.s, 1);
  const Mag p1 = mul_hi(X.re, y.m);
  const Mag p2 = mul_hi(X.im, yp);
  const uint32_t s1 = (X.signs & kSignBit) ^ y.s;
  const uint32_t s2 = ((X.signs << 1) & kSignBit) ^ sp ^ (c == 0 ? kSignBit : 0u);
  uint32_t s;
  const Mag r = signed_add(p1, s1, p2, s2, s);
  if (!Norm) return WV{r, s, X.e + y.e + 128};
  return normalize_pair(WV{r, s, X.e + y.e + 128});
}

// P * Q, both split over the pair, not normalised (a final product):
//   re lane: P.re Q.re - P.im Q.im      im lane: P.im Q.re + P.re Q.im
__device__ __forceinline__ WV mul_pair(const WV &P, const WV &Q, int c) {
  const Mag Pp = shfl_xor_mag(P.m, 1), Qp = shfl_xor_mag(Q.m, 1);
  const uint32_t sPp = __shfl_xor_sync(0xffffffffu, P.s, 1), sQp = __shfl_xor_sync(0xffffffffu, Q.s, 1);
  const bool re = c == 0;
  // re: (P.m, Q.m) - (Pp, Qp); im: (P.m, Qp) + (Pp, Q.m)
  const Mag b1 = re ? Q.m : Qp, b2 = re ? Qp : Q.m;
  const uint32_t sb1 = re ? Q.s : sQp, sb2 = re ? sQp : Q.s;
  const Mag p1 = mul_hi(P.m, b1);
  const Mag p2 = mul_hi(Pp, b2);
  uint32_t s;
  const Mag r = signed_add(p1, P.s ^ sb1, p2, sPp ^ sb2 ^ (re ? kSignBit : 0u), s);
  return WV{r, s, P.e + Q.e + 128};
}

// Multiply by a small integer 1 <= k <= 256: (m >> 8) * k, exponent + 8.
__device__ __forceinline__ WV mul_small(const WV &v, uint32_t k) {
  const Mag a = shr(v.m, 8);
  uint32_t r0, r1, r2, r3;
  asm("{\n\t"
      "mul.lo.u32      %0, %4, %8;\n\t"
      "mul.hi.u32      %1, %4, %8;\n\t"
      "mad.lo.cc.u32   %1, %5, %8, %1;\n\t"
      "madc.hi.u32     %2, %5, %8, 0;\n\t"
      "mad.lo.cc.u32   %2, %6, %8, %2;\n\t"
      "madc.hi.u32     %3, %6, %8, 0;\n\t"
      "mad.lo.u32      %3, %7, %8, %3;\n\t"
      "}"
      : "=&r"(r0), "=&r"(r1), "=&r"(r2), "=&r"(r3)
      : "r"(a.w0), "r"(a.w1), "r"(a.w2), "r"(a.w3), "r"(k));
  return WV{Mag{r0, r1, r2, r3}, v.s, v.e + 8};
}

// A double from a 53-bit integer significand (bit 52 set, or zero) and the
// binary exponent of its least significant bit; flushes to zero below the
// normal range and saturates to infinity above it.
__device__ __forceinline__ double make_double(unsigned long long sig, int lsb_exp, uint32_t sign) {
  const int field = lsb_exp + 52 + 1023;
  const unsigned long long sbit = static_cast<unsigned long long>(sign) << 32;
  if (sig == 0ULL || field <= 0) return __longlong_as_double(static_cast<long long>(sbit));
  if (field >= 2047) return __longlong_as_double(static_cast<long long>(sbit | 0x7ff0000000000000ULL));
  const unsigned long long bits = sbit |
                                  (static_cast<unsigned long long>(field) << 52) | (sig & 0x000fffffffffffffULL);
  return __longlong_as_double(static_cast<long long>(bits));
}

// Top 53 bits of m below (and including) bit position `top` (0-based), as an
// integer; bits above `top` must be zero.
__device__ __forceinline__ unsigned long long bits53(const Mag &m, int top) {
  // shift so that bit `top` lands on bit 52 of a 64-bit word
  const int sh = top - 52;
  Mag x = sh >= 0 ? shr(m, sh) : shl(m, -sh);
  return (static_cast<unsigned long long>(x.w1) << 32) | x.w0;
}

// A lane value as a double-double (truncated to 106 bits; not renormalised).
// Fast path for a leading bit in the top limb: the value shifted so that the
// leading bit is bit 127 gives the 53 bits of the high word and the next 53
// bits of the low word directly.
__device__ __forceinline__ dd to_dd_general(const WV &v);
__device__ __forceinline__ dd to_dd(const WV &v) {
  if (v.m.w3 == 0u) return to_dd_general(v);
  const int s = __clz(static_cast<int>(v.m.w3));  // 0..31
  const uint32_t t3 = __funnelshift_l(v.m.w2, v.m.w3, s), t2 = __funnelshift_l(v.m.w1, v.m.w2, s);
  const uint32_t t1 = __funnelshift_l(v.m.w0, v.m.w1, s), t0 = v.m.w0 << s;
  const unsigned long long top64 = (static_cast<unsigned long long>(t3) << 32) | t2;
  const unsigned long long low64 = (static_cast<unsigned long long>(t1) << 32) | t0;
  const unsigned long long hs = top64 >> 11;                              // bits 127..75
  const unsigned long long ls = ((top64 & 0x7ffULL) << 42) | (low64 >> 22);  // bits 74..22
  // value = m 2^e with bit 127 of (m << s) the leading bit: hi lsb at 2^(e + 75 - s)
  const double hi = make_double(hs, v.e + 75 - s, v.s);
  if (ls == 0ULL) return dd{hi, 0.0};
  const int lz = __clzll(static_cast<long long>(ls)) - 11;  // leading zeros of the 53-bit field
  const double lo = make_double(ls << lz, v.e + 22 - s - lz, v.s);
  return dd{hi, lo};
}

__device__ __forceinline__ dd to_dd_general(const WV &v) {
  const int lz = clz128(v.m);
  if (lz == 128) return dd{0.0, 0.0};
  const int top = 127 - lz;
  const unsigned long long h = bits53(v.m, top);
  const double hi = make_double(h, v.e + top - 52, v.s);
  // remainder below the 53 leading bits
  Mag r = v.m;
  const Mag hm = shl(Mag{static_cast<uint32_t>(h), static_cast<uint32_t>(h >> 32), 0u, 0u}, top - 52 >= 0 ? top - 52 : 0);
  if (top - 52 >= 0) {
    asm("{\n\t"
        "sub.cc.u32  %0, %0, %4;\n\t"
        "subc.cc.u32 %1, %1, %5;\n\t"
        "subc.cc.u32 %2, %2, %6;\n\t"
        "subc.u32    %3, %3, %7;\n\t"
        "}"
        : "+r"(r.w0), "+r"(r.w1), "+r"(r.w2), "+r"(r.w3)
        : "r"(hm.w0), "r"(hm.w1), "r"(hm.w2), "r"(hm.w3));
  } else {
    r = Mag{0u, 0u, 0u, 0u};
  }
  const int lz2 = clz128(r);
  if (lz2 == 128) return dd{hi, 0.0};
  const int top2 = 127 - lz2;
  const double lo = make_double(bits53(r, top2), v.e + top2 - 52, v.s);
  return dd{hi, lo};
}

// ---------------------------------------------------------------------------
// conversion of a complex double-double to the block format (exact up to
// truncation below 2^-125 of the larger component)
// ---------------------------------------------------------------------------

struct Comp {  // a real double-double as sign and 128-bit magnitude times 2^e
  Mag m;
  uint32_t s;
  int32_t e;
};

__device__ __forceinline__ void split_double(double d, uint32_t &s, unsigned long long &M, int &X) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(d));
  s = static_cast<uint32_t>(b >> 32) & kSignBit;
  const int ef = static_cast<int>((b >> 52) & 0x7ff);
  const unsigned long long f = b & 0x000fffffffffffffULL;
  if (ef == 0) {
    M = f;
    X = -1074;
  } else {
    M = f | 0x0010000000000000ULL;
    X = ef - 1075;
  }
}

__device__ __forceinline__ Mag mag_from_u64(unsigned long long v) {
  return Mag{static_cast<uint32_t>(v), static_cast<uint32_t>(v >> 32), 0u, 0u};
}

// hi + lo (|lo| <= ulp(hi)) as sign-magnitude with the leading bit of hi at
// position 124.
__device__ __forceinline__ Comp comp_from_dd(double hi, double lo) {
  uint32_t sh_, sl_;
  unsigned long long Mh, Ml;
  int Xh, Xl;
  split_double(hi, sh_, Mh, Xh);
  split_double(lo, sl_, Ml, Xl);
  if (Mh == 0ULL) {
    if (Ml == 0ULL) return Comp{Mag{0u, 0u, 0u, 0u}, 0u, kZeroExp};
    // a lone low word: treat it as the high word
    Mh = Ml;
    Xh = Xl;
    sh_ = sl_;
    Ml = 0ULL;
  }
  const int lzh = __clzll(static_cast<long long>(Mh));  // 11 for a normal number
  const int Ec = Xh - (124 - (63 - lzh));  // exponent of bit 0 when Mh's top bit sits at 124
  Mag a = shl(mag_from_u64(Mh), 124 - (63 - lzh));
  if (Ml != 0ULL) {
    const int sl = Xl - Ec;  // shift of Ml relative to bit 0
    Mag b = sl >= 0 ? shl(mag_from_u64(Ml), sl) : shr(mag_from_u64(Ml), -sl);
    uint32_t s;
    a = signed_add(a, sh_, b, sl_, s);
    sh_ = s;
  }
  return Comp{a, sh_, Ec};
}

// A complex double-double as a normalised full value.  Each component is
// first renormalised (|lo| <= ulp(hi)/2) so that any input double-double is
// accepted.
__device__ __forceinline__ WF wf_from_cdd(double rh, double rl, double ih, double il) {
  double rs, re_, is_, ie_;
  two_sum(rh, rl, rs, re_);
  two_sum(ih, il, is_, ie_);
  Comp r = comp_from_dd(rs, re_), i = comp_from_dd(is_, ie_);
  const bool rz = is_zero(r.m), iz = is_zero(i.m);
  if (rz && iz) return WF{Mag{0u, 0u, 0u, 0u}, Mag{0u, 0u, 0u, 0u}, 0u, kZeroExp};
  int e;
  if (rz) {
    e = i.e;
  } else if (iz) {
    e = r.e;
  } else {
    e = max(r.e, i.e);
  }
  const Mag rm = rz ? r.m : shr(r.m, e - r.e);
  const Mag im = iz ? i.m : shr(i.m, e - i.e);
  // normalise: the larger magnitude to [2^125, 2^126)
  const int z = min(clz128(rm), clz128(im));
  const int sh = z - 2;
  WF out;
  out.re = sh >= 0 ? shl(rm, sh) : shr(rm, -sh);
  out.im = sh >= 0 ? shl(im, sh) : shr(im, -sh);
  out.e = e - sh;
  out.signs = (r.s & kSignBit) | ((i.s & kSignBit) >> 1);
  return out;
}

// Full complex product (one thread holds both components), normalised.
__device__ __forceinline__ WF wf_mul(const WF &x, const WF &y) {
  const uint32_t xr = x.signs & kSignBit, xi = (x.signs << 1) & kSignBit;
  const uint32_t yr = y.signs & kSignBit, yi = (y.signs << 1) & kSignBit;
  uint32_t sre, sim;
  const Mag re = signed_add(mul_hi(x.re, y.re), xr ^ yr, mul_hi(x.im, y.im), xi ^ yi ^ kSignBit, sre);
  const Mag im = signed_add(mul_hi(x.re, y.im), xr ^ yi, mul_hi(x.im, y.re), xi ^ yr, sim);
  if (is_zero(re) && is_zero(im)) return WF{Mag{0u, 0u, 0u, 0u}, Mag{0u, 0u, 0u, 0u}, 0u, kZeroExp};
  const int sh = min(clz128(re), clz128(im)) - 2;
  WF out;
  out.re = sh >= 0 ? shl(re, sh) : shr(re, -sh);
  out.im = sh >= 0 ? shl(im, sh) : shr(im, -sh);
  out.e = x.e + y.e + 128 - sh;
  out.signs = (sre & kSignBit) | ((sim & kSignBit) >> 1);
  return out;
}

}  // namespace wide
}  // namespace pe
