// Complex block floating point with 256-bit mantissas and 224-bit
// accumulators, on the integer pipes: the arithmetic of the quad-double
// evaluation (precision PE_QD_INT).
//
// Values.  A complex number is (A + iB) * 2^e with A and B in sign-magnitude
// form: a 256-bit magnitude in eight 32-bit limbs (limb 0 least significant)
// and a sign bit each, and one shared 32-bit exponent e.  Values that feed
// further products are normalised: max(|A|, |B|) in [2^253, 2^254); zero is
// all-zero magnitudes with e = kZeroExp.  A product keeps the top 256 bits of
// the 512-bit product of the magnitudes, computed from the partial products of
// columns 8..14 and the high words of column 7; the dropped part is below 16
// units of the result's last place, so one product errs by about 2^-246
// relative to the product of the operands' magnitudes -- the normwise
// measure of the evaluation -- against 2^-209 or so for quad-double
// arithmetic.
//
// Lane pairs: lanes 2q and 2q+1 hold the real and the imaginary part of the
// values of point q (one magnitude and sign per lane, the exponent on both).
//
// Sums.  Each output component is summed in an accumulator of its own: a
// 224-bit two's complement integer A (seven limbs) and an exponent, value
// A * 2^e, with |A| < 2^221 between additions.  A term is aligned to the
// larger of the two exponents (the bits shifted out of the smaller one are
// dropped), added, and the accumulator is shifted right by two when it
// leaves the headroom.  Every addition errs by at most a unit of 2^e, about
// 2^-219 relative to the largest term so far.  The accumulator occupies the
// 32 bytes the output component takes as a quad-double (limbs 0..6, then e),
// so the sums run in place in the output arrays; a final pass rounds each one
// to a quad-double.
#pragma once

#include <cstdint>

#include "wide.cuh"

namespace pe {
namespace qd {

constexpr int L = 8;  // limbs of a magnitude
constexpr int LA = 7; // limbs of an accumulator
constexpr int32_t kZeroExp = -(1 << 28);
constexpr uint32_t kSignBit = 0x80000000u;

struct Mag {
  uint32_t w[L];
};

// One component held by a lane: magnitude, sign (0 or kSignBit), exponent.
struct WV {
  Mag m;
  uint32_t s;
  int32_t e;
};

// A full complex value as stored in memory: 20 words (80 bytes): re limbs,
// im limbs, signs (bit 31 re, bit 30 im), exponent, 2 spare.
struct WF {
  Mag re, im;
  uint32_t signs;
  int32_t e;
};

// A sum: 224-bit two's complement integer and the exponent of its bit 0.
struct Acc {
  uint32_t w[LA];
  int32_t e;
};

__device__ __forceinline__ Mag zero_mag() {
  Mag z;
#pragma unroll
  for (int i = 0; i < L; i++) z.w[i] = 0u;
  return z;
}

__device__ __forceinline__ bool is_zero(const Mag &a) {
  uint32_t o = 0u;
#pragma unroll
  for (int i = 0; i < L; i++) o |= a.w[i];
  return o == 0u;
}

__device__ __forceinline__ WF load_wf(const uint32_t *p) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
  const uint4 a = __ldg(q), b = __ldg(q + 1), c = __ldg(q + 2), d = __ldg(q + 3);
  const uint2 x = __ldg(reinterpret_cast<const uint2 *>(q + 4));
  return WF{Mag{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}}, Mag{{c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w}}, x.x,
            static_cast<int32_t>(x.y)};
}

__device__ __forceinline__ WF load_wf_coherent(const uint32_t *p) {
  const uint4 *q = reinterpret_cast<const uint4 *>(p);
  const uint4 a = q[0], b = q[1], c = q[2], d = q[3];
  const uint2 x = *reinterpret_cast<const uint2 *>(q + 4);
  return WF{Mag{{a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w}}, Mag{{c.x, c.y, c.z, c.w, d.x, d.y, d.z, d.w}}, x.x,
            static_cast<int32_t>(x.y)};
}

__device__ __forceinline__ void store_wf(uint32_t *p, const WF &v) {
  uint4 *q = reinterpret_cast<uint4 *>(p);
  q[0] = make_uint4(v.re.w[0], v.re.w[1], v.re.w[2], v.re.w[3]);
  q[1] = make_uint4(v.re.w[4], v.re.w[5], v.re.w[6], v.re.w[7]);
  q[2] = make_uint4(v.im.w[0], v.im.w[1], v.im.w[2], v.im.w[3]);
  q[3] = make_uint4(v.im.w[4], v.im.w[5], v.im.w[6], v.im.w[7]);
  q[4] = make_uint4(v.signs, static_cast<uint32_t>(v.e), 0u, 0u);
}

// The component c (0 real, 1 imaginary) of a full value, as a lane value.
__device__ __forceinline__ WV component(const WF &x, int c) {
  const bool re = c == 0;
  WV v;
#pragma unroll
  for (int i = 0; i < L; i++) v.m.w[i] = re ? x.re.w[i] : x.im.w[i];
  v.s = (re ? x.signs : (x.signs << 1)) & kSignBit;
  v.e = x.e;
  return v;
}

// ---------------------------------------------------------------------------
// multiply-accumulate steps (each carry chain inside one asm statement)
// ---------------------------------------------------------------------------

// (w2:w1:w0) += a * b
__device__ __forceinline__ void mac3(uint32_t &w0, uint32_t &w1, uint32_t &w2, uint32_t a, uint32_t b) {
  asm("mad.lo.cc.u32   %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32  %1, %3, %4, %1;\n\t"
      "addc.u32        %2, %2, 0;"
      : "+r"(w0), "+r"(w1), "+r"(w2)
      : "r"(a), "r"(b));
}

// (w1:w0) += a * b, no carry out of w1 (the caller knows there is none)
__device__ __forceinline__ void mac2(uint32_t &w0, uint32_t &w1, uint32_t a, uint32_t b) {
  asm("mad.lo.cc.u32   %0, %2, %3, %0;\n\t"
      "madc.hi.u32     %1, %2, %3, %1;"
      : "+r"(w0), "+r"(w1)
      : "r"(a), "r"(b));
}

// (w1:w0) += hi(a * b)
__device__ __forceinline__ void machi2(uint32_t &w0, uint32_t &w1, uint32_t a, uint32_t b) {
  asm("mad.hi.cc.u32   %0, %2, %3, %0;\n\t"
      "addc.u32        %1, %1, 0;"
      : "+r"(w0), "+r"(w1)
      : "r"(a), "r"(b));
}

// Top 256 bits of the 512-bit product a*b, low by less than 16 units in the
// last place: column words 8..15 of the product scan, with the high words of
// column 7 and nothing below.
__device__ __forceinline__ Mag mul_hi(const Mag &a, const Mag &b) {
  uint32_t C[L + 1];
#pragma unroll
  for (int i = 0; i <= L; i++) C[i] = 0u;
#pragma unroll
  for (int i = 0; i < L; i++) machi2(C[0], C[1], a.w[i], b.w[L - 1 - i]);
#pragma unroll
  for (int c = L; c <= 2 * L - 2; c++) {
#pragma unroll
    for (int i = c - (L - 1); i <= L - 1; i++) {
      if (c == 2 * L - 2)
        mac2(C[c - L], C[c - L + 1], a.w[i], b.w[c - i]);
      else
        mac3(C[c - L], C[c - L + 1], C[c - L + 2], a.w[i], b.w[c - i]);
    }
  }
  Mag r;
#pragma unroll
  for (int i = 0; i < L; i++) r.w[i] = C[i];
  return r;
}

// r = a + (b ^ m) + (m & 1) over eight limbs; returns the carry out.  With
// m = 0 this is a + b, with m = ~0 it is a - b (mod 2^256).
__device__ __forceinline__ uint32_t add_xor(Mag &r, const Mag &a, const Mag &b, uint32_t m) {
  Mag x;
#pragma unroll
  for (int i = 0; i < L; i++) x.w[i] = b.w[i] ^ m;
  uint32_t cout;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "and.b32         t, %25, 1;\n\t"
      "add.cc.u32      t, t, 0xffffffff;\n\t"  // carry-in = m & 1
      "addc.cc.u32     %0, %9, %17;\n\t"
      "addc.cc.u32     %1, %10, %18;\n\t"
      "addc.cc.u32     %2, %11, %19;\n\t"
      "addc.cc.u32     %3, %12, %20;\n\t"
      "addc.cc.u32     %4, %13, %21;\n\t"
      "addc.cc.u32     %5, %14, %22;\n\t"
      "addc.cc.u32     %6, %15, %23;\n\t"
      "addc.cc.u32     %7, %16, %24;\n\t"
      "addc.u32        %8, 0, 0;\n\t"
      "}"
      : "=&r"(r.w[0]), "=&r"(r.w[1]), "=&r"(r.w[2]), "=&r"(r.w[3]), "=&r"(r.w[4]), "=&r"(r.w[5]), "=&r"(r.w[6]),
        "=&r"(r.w[7]), "=&r"(cout)
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(a.w[5]), "r"(a.w[6]), "r"(a.w[7]),
        "r"(x.w[0]), "r"(x.w[1]), "r"(x.w[2]), "r"(x.w[3]), "r"(x.w[4]), "r"(x.w[5]), "r"(x.w[6]), "r"(x.w[7]),
        "r"(m));
  return cout;
}

// r = (r ^ m) + (m & 1): two's complement negation when m = ~0.
__device__ __forceinline__ void neg_if(Mag &r, uint32_t m) {
#pragma unroll
  for (int i = 0; i < L; i++) r.w[i] ^= m;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "and.b32         t, %8, 1;\n\t"
      "add.cc.u32      t, t, 0xffffffff;\n\t"
      "addc.cc.u32     %0, %0, 0;\n\t"
      "addc.cc.u32     %1, %1, 0;\n\t"
      "addc.cc.u32     %2, %2, 0;\n\t"
      "addc.cc.u32     %3, %3, 0;\n\t"
      "addc.cc.u32     %4, %4, 0;\n\t"
      "addc.cc.u32     %5, %5, 0;\n\t"
      "addc.cc.u32     %6, %6, 0;\n\t"
      "addc.u32        %7, %7, 0;\n\t"
      "}"
      : "+r"(r.w[0]), "+r"(r.w[1]), "+r"(r.w[2]), "+r"(r.w[3]), "+r"(r.w[4]), "+r"(r.w[5]), "+r"(r.w[6]),
        "+r"(r.w[7])
      : "r"(m));
}

// (p1 with sign s1) + (p2 with sign s2), magnitudes below 2^255: magnitude
// and sign of the sum.
__device__ __forceinline__ Mag signed_add(const Mag &p1, uint32_t s1, const Mag &p2, uint32_t s2, uint32_t &s) {
  const uint32_t m = static_cast<uint32_t>(static_cast<int32_t>(s1 ^ s2) >> 31);  // all ones: subtract
  Mag r;
  const uint32_t cout = add_xor(r, p1, p2, m);
  // subtracting and no carry out: p2 > p1, negate the difference
  const uint32_t nm = m & (cout - 1u);
  neg_if(r, nm);
  s = nm ? s2 : s1;
  return r;
}

// ---------------------------------------------------------------------------
// shifts
// ---------------------------------------------------------------------------

// Leading zeros of a 256-bit magnitude (256 for zero).
__device__ __forceinline__ int clz256(const Mag &a) {
  int z = 256;
#pragma unroll
  for (int i = 0; i < L; i++)
    if (a.w[i]) z = (L - 1 - i) * 32 + __clz(static_cast<int>(a.w[i]));
  return z;
}

template <int S>
__device__ __forceinline__ void words_up(Mag &x, bool on) {  // x <<= 32 S when on
#pragma unroll
  for (int i = L - 1; i >= 0; i--) x.w[i] = on ? (i >= S ? x.w[i - S] : 0u) : x.w[i];
}

template <int S>
__device__ __forceinline__ void words_down(Mag &x, bool on) {  // x >>= 32 S when on
#pragma unroll
  for (int i = 0; i < L; i++) x.w[i] = on ? (i + S < L ? x.w[i + S] : 0u) : x.w[i];
}

// Left shift by 0 <= n < 256.
__device__ __forceinline__ Mag shl(const Mag &a, int n) {
  Mag x = a;
  words_up<4>(x, (n & 128) != 0);
  words_up<2>(x, (n & 64) != 0);
  words_up<1>(x, (n & 32) != 0);
  const int b = n & 31;
  Mag r;
#pragma unroll
  for (int i = L - 1; i > 0; i--) r.w[i] = __funnelshift_l(x.w[i - 1], x.w[i], b);
  r.w[0] = x.w[0] << b;
  return r;
}

// Right shift by n >= 0 (n >= 256 gives zero).
__device__ __forceinline__ Mag shr(const Mag &a, int n) {
  if (n >= 256) return zero_mag();
  Mag x = a;
  words_down<4>(x, (n & 128) != 0);
  words_down<2>(x, (n & 64) != 0);
  words_down<1>(x, (n & 32) != 0);
  const int b = n & 31;
  Mag r;
#pragma unroll
  for (int i = 0; i < L - 1; i++) r.w[i] = __funnelshift_r(x.w[i], x.w[i + 1], b);
  r.w[L - 1] = x.w[L - 1] >> b;
  return r;
}

__device__ __forceinline__ Mag shfl_xor_mag(const Mag &a, int m) {
  Mag r;
#pragma unroll
  for (int i = 0; i < L; i++) r.w[i] = __shfl_xor_sync(0xffffffffu, a.w[i], m);
  return r;
}

// Normalise a lane-pair value: the larger magnitude of the pair to
// [2^253, 2^254), both lanes shifted alike; zero pairs get kZeroExp.
__device__ __forceinline__ WV normalize_pair(const WV &v) {
  // usual case: both leading bits in the top limb, a left shift below 30
  const int lz7 = __clz(static_cast<int>(v.m.w[L - 1]));
  const int z7 = min(lz7, __shfl_xor_sync(0xffffffffu, lz7, 1));
  if (__all_sync(0xffffffffu, z7 >= 2 && z7 < 32)) {
    const int sh = z7 - 2;
    WV r;
#pragma unroll
    for (int i = L - 1; i > 0; i--) r.m.w[i] = __funnelshift_l(v.m.w[i - 1], v.m.w[i], sh);
    r.m.w[0] = v.m.w[0] << sh;
    r.s = v.s;
    r.e = v.e - sh;
    return r;
  }
  const int lz = clz256(v.m);
  const int z = min(lz, __shfl_xor_sync(0xffffffffu, lz, 1));
  if (z == 256) return WV{zero_mag(), 0u, kZeroExp};
  const int sh = z - 2;  // leading bit to position 253
  if (sh >= 0) return WV{shl(v.m, sh), v.s, v.e - sh};
  return WV{shr(v.m, -sh), v.s, v.e - sh};
}

// y (split over the pair) times X (full value on both lanes), normalised:
//   re: X.re y.re - X.im y.im      im: X.re y.im + X.im y.re
__device__ __forceinline__ WV mul_x(const WV &y, const WF &X, int c) {
  const Mag yp = shfl_xor_mag(y.m, 1);
  const uint32_t sp = __shfl_xor_sync(0xffffffffu, y.s, 1);
  const Mag p1 = mul_hi(X.re, y.m);
  const Mag p2 = mul_hi(X.im, yp);
  const uint32_t s1 = (X.signs & kSignBit) ^ y.s;
  const uint32_t s2 = ((X.signs << 1) & kSignBit) ^ sp ^ (c == 0 ? kSignBit : 0u);
  uint32_t s;
  const Mag r = signed_add(p1, s1, p2, s2, s);
  return normalize_pair(WV{r, s, X.e + y.e + 256});
}

// P * Q, both split over the pair, not normalised (a final product):
//   re lane: P.re Q.re - P.im Q.im      im lane: P.im Q.re + P.re Q.im
__device__ __forceinline__ WV mul_pair(const WV &P, const WV &Q, int c) {
  const Mag Pp = shfl_xor_mag(P.m, 1), Qp = shfl_xor_mag(Q.m, 1);
  const uint32_t sPp = __shfl_xor_sync(0xffffffffu, P.s, 1), sQp = __shfl_xor_sync(0xffffffffu, Q.s, 1);
  const bool re = c == 0;
  Mag b1, b2;
#pragma unroll
  for (int i = 0; i < L; i++) {
    b1.w[i] = re ? Q.m.w[i] : Qp.w[i];
    b2.w[i] = re ? Qp.w[i] : Q.m.w[i];
  }
  const uint32_t sb1 = re ? Q.s : sQp, sb2 = re ? sQp : Q.s;
  const Mag p1 = mul_hi(P.m, b1);
  const Mag p2 = mul_hi(Pp, b2);
  uint32_t s;
  const Mag r = signed_add(p1, P.s ^ sb1, p2, sPp ^ sb2 ^ (re ? kSignBit : 0u), s);
  return WV{r, s, P.e + Q.e + 256};
}

// Multiply by a small integer 1 <= k <= 256: (m >> 8) * k, exponent + 8.
__device__ __forceinline__ WV mul_small(const WV &v, uint32_t k) {
  const Mag a = shr(v.m, 8);
  Mag r = zero_mag();
  // row product: r = a * k, one carry chain
  asm("{\n\t"
      "mul.lo.u32      %0, %8, %16;\n\t"
      "mul.hi.u32      %1, %8, %16;\n\t"
      "mad.lo.cc.u32   %1, %9, %16, %1;\n\t"
      "madc.hi.u32     %2, %9, %16, 0;\n\t"
      "mad.lo.cc.u32   %2, %10, %16, %2;\n\t"
      "madc.hi.u32     %3, %10, %16, 0;\n\t"
      "mad.lo.cc.u32   %3, %11, %16, %3;\n\t"
      "madc.hi.u32     %4, %11, %16, 0;\n\t"
      "mad.lo.cc.u32   %4, %12, %16, %4;\n\t"
      "madc.hi.u32     %5, %12, %16, 0;\n\t"
      "mad.lo.cc.u32   %5, %13, %16, %5;\n\t"
      "madc.hi.u32     %6, %13, %16, 0;\n\t"
      "mad.lo.cc.u32   %6, %14, %16, %6;\n\t"
      "madc.hi.u32     %7, %14, %16, 0;\n\t"
      "mad.lo.u32      %7, %15, %16, %7;\n\t"
      "}"
      : "=&r"(r.w[0]), "=&r"(r.w[1]), "=&r"(r.w[2]), "=&r"(r.w[3]), "=&r"(r.w[4]), "=&r"(r.w[5]), "=&r"(r.w[6]),
        "=&r"(r.w[7])
      : "r"(a.w[0]), "r"(a.w[1]), "r"(a.w[2]), "r"(a.w[3]), "r"(a.w[4]), "r"(a.w[5]), "r"(a.w[6]), "r"(a.w[7]),
        "r"(k));
  return WV{r, v.s, v.e + 8};
}

// Full complex product (one thread holds both components), normalised.
__device__ __forceinline__ WF wf_mul(const WF &x, const WF &y) {
  const uint32_t xr = x.signs & kSignBit, xi = (x.signs << 1) & kSignBit;
  const uint32_t yr = y.signs & kSignBit, yi = (y.signs << 1) & kSignBit;
  uint32_t sre, sim;
  const Mag re = signed_add(mul_hi(x.re, y.re), xr ^ yr, mul_hi(x.im, y.im), xi ^ yi ^ kSignBit, sre);
  const Mag im = signed_add(mul_hi(x.re, y.im), xr ^ yi, mul_hi(x.im, y.re), xi ^ yr, sim);
  if (is_zero(re) && is_zero(im)) return WF{zero_mag(), zero_mag(), 0u, kZeroExp};
  const int sh = min(clz256(re), clz256(im)) - 2;
  WF out;
  out.re = sh >= 0 ? shl(re, sh) : shr(re, -sh);
  out.im = sh >= 0 ? shl(im, sh) : shr(im, -sh);
  out.e = x.e + y.e + 256 - sh;
  out.signs = (sre & kSignBit) | ((sim & kSignBit) >> 1);
  return out;
}

// ---------------------------------------------------------------------------
// conversion of a complex quad-double to the block format
// ---------------------------------------------------------------------------

struct Comp {  // a real number as sign and 256-bit magnitude times 2^e
  Mag m;
  uint32_t s;
  int32_t e;
};

__device__ __forceinline__ Mag mag_from_u64(unsigned long long v) {
  Mag r = zero_mag();
  r.w[0] = static_cast<uint32_t>(v);
  r.w[1] = static_cast<uint32_t>(v >> 32);
  return r;
}

// x0 + ... + x_{NP-1} for any NP <= 8 finite doubles (overlapping,
// unnormalised or of mixed signs), as sign and magnitude with the leading bit
// of the largest part at position 250.  Bits below position 0 are dropped (at
// most NP units of 2^-250 relative to the largest part).
template <int NP>
__device__ __forceinline__ Comp comp_from_parts(const double x[NP]) {
  static_assert(NP >= 1 && NP <= 8, "the sum must stay below 2^255");
  uint32_t s[NP];
  unsigned long long M[NP];
  int X[NP];
  int top = INT32_MIN;
#pragma unroll
  for (int i = 0; i < NP; i++) {
    wide::split_double(x[i], s[i], M[i], X[i]);
    if (M[i]) top = max(top, X[i] + 63 - __clzll(static_cast<long long>(M[i])));
  }
  if (top == INT32_MIN) return Comp{zero_mag(), 0u, kZeroExp};
  const int base = top - 250;  // exponent of bit 0
  Mag acc = zero_mag();        // two's complement
#pragma unroll
  for (int i = 0; i < NP; i++) {
    if (!M[i]) continue;
    const int pos = X[i] - base;  // position of the significand's bit 0
    const Mag v = pos >= 0 ? shl(mag_from_u64(M[i]), pos) : shr(mag_from_u64(M[i]), -pos);
    Mag r;
    add_xor(r, acc, v, s[i] ? 0xffffffffu : 0u);
    acc = r;
  }
  const uint32_t neg = static_cast<uint32_t>(static_cast<int32_t>(acc.w[L - 1]) >> 31);
  neg_if(acc, neg);
  return Comp{acc, neg & kSignBit, base};
}

__device__ __forceinline__ Comp comp_from_qd(const double x[4]) { return comp_from_parts<4>(x); }

// A complex quad-double (re0..re3, im0..im3) as a normalised full value.
__device__ __forceinline__ WF wf_from_cqd(const double *v) {
  const Comp r = comp_from_qd(v), i = comp_from_qd(v + 4);
  const bool rz = is_zero(r.m), iz = is_zero(i.m);
  if (rz && iz) return WF{zero_mag(), zero_mag(), 0u, kZeroExp};
  const int e = rz ? i.e : iz ? r.e : max(r.e, i.e);
  const Mag rm = rz ? r.m : shr(r.m, e - r.e);
  const Mag im = iz ? i.m : shr(i.m, e - i.e);
  const int sh = min(clz256(rm), clz256(im)) - 2;
  WF out;
  out.re = sh >= 0 ? shl(rm, sh) : shr(rm, -sh);
  out.im = sh >= 0 ? shl(im, sh) : shr(im, -sh);
  out.e = e - sh;
  out.signs = (r.s & kSignBit) | ((i.s & kSignBit) >> 1);
  return out;
}

// ---------------------------------------------------------------------------
// accumulators
// ---------------------------------------------------------------------------

__device__ __forceinline__ Acc acc_zero() {
  Acc a;
#pragma unroll
  for (int i = 0; i < LA; i++) a.w[i] = 0u;
  a.e = kZeroExp;
  return a;
}

__device__ __forceinline__ bool acc_is_zero(const Acc &a) {
  uint32_t o = 0u;
#pragma unroll
  for (int i = 0; i < LA; i++) o |= a.w[i];
  return o == 0u;
}

// 32 bytes: limbs 0..6, exponent.
__device__ __forceinline__ Acc load_acc(const double *p) {
  const uint4 a = reinterpret_cast<const uint4 *>(p)[0], b = reinterpret_cast<const uint4 *>(p)[1];
  return Acc{{a.x, a.y, a.z, a.w, b.x, b.y, b.z}, static_cast<int32_t>(b.w)};
}

__device__ __forceinline__ void store_acc(double *p, const Acc &a) {
  reinterpret_cast<uint4 *>(p)[0] = make_uint4(a.w[0], a.w[1], a.w[2], a.w[3]);
  reinterpret_cast<uint4 *>(p)[1] = make_uint4(a.w[4], a.w[5], a.w[6], static_cast<uint32_t>(a.e));
}

// Arithmetic right shift of the accumulator's integer by n >= 0 (n >= 223
// leaves only the sign).
__device__ __forceinline__ void acc_sar(Acc &a, int n) {
  n = min(n, 223);
  const uint32_t fill = static_cast<uint32_t>(static_cast<int32_t>(a.w[LA - 1]) >> 31);
  const bool s4 = (n & 128) != 0, s2 = (n & 64) != 0, s1 = (n & 32) != 0;
#pragma unroll
  for (int i = 0; i < LA; i++) a.w[i] = s4 ? (i + 4 < LA ? a.w[i + 4] : fill) : a.w[i];
#pragma unroll
  for (int i = 0; i < LA; i++) a.w[i] = s2 ? (i + 2 < LA ? a.w[i + 2] : fill) : a.w[i];
#pragma unroll
  for (int i = 0; i < LA; i++) a.w[i] = s1 ? (i + 1 < LA ? a.w[i + 1] : fill) : a.w[i];
  const int b = n & 31;
#pragma unroll
  for (int i = 0; i < LA - 1; i++) a.w[i] = __funnelshift_r(a.w[i], a.w[i + 1], b);
  a.w[LA - 1] = static_cast<uint32_t>(static_cast<int32_t>(a.w[LA - 1]) >> b);
}

// a.w += (x ^ m) + (m & 1) over seven limbs (x a magnitude; m = ~0 subtracts).
__device__ __forceinline__ void acc_add_raw(Acc &a, const uint32_t x[LA], uint32_t m) {
  uint32_t y[LA];
#pragma unroll
  for (int i = 0; i < LA; i++) y[i] = x[i] ^ m;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "and.b32         t, %14, 1;\n\t"
      "add.cc.u32      t, t, 0xffffffff;\n\t"
      "addc.cc.u32     %0, %0, %7;\n\t"
      "addc.cc.u32     %1, %1, %8;\n\t"
      "addc.cc.u32     %2, %2, %9;\n\t"
      "addc.cc.u32     %3, %3, %10;\n\t"
      "addc.cc.u32     %4, %4, %11;\n\t"
      "addc.cc.u32     %5, %5, %12;\n\t"
      "addc.u32        %6, %6, %13;\n\t"
      "}"
      : "+r"(a.w[0]), "+r"(a.w[1]), "+r"(a.w[2]), "+r"(a.w[3]), "+r"(a.w[4]), "+r"(a.w[5]), "+r"(a.w[6])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(m));
}

// Keep |A| < 2^221: when bits 223..221 are not all equal, shift right by 2.
__device__ __forceinline__ void acc_headroom(Acc &a) {
  const int32_t top = static_cast<int32_t>(a.w[LA - 1]);
  const bool out = ((top >> 29) != (top >> 31));
  if (out) {
#pragma unroll
    for (int i = 0; i < LA - 1; i++) a.w[i] = __funnelshift_r(a.w[i], a.w[i + 1], 2);
    a.w[LA - 1] = static_cast<uint32_t>(top >> 2);
    a.e += 2;
  }
}

// a += t for a lane term t (magnitude below 2^254).  The term's lowest limb
// is dropped (t = (m >> 32) 2^(e + 32), below 2^222), then the operand with
// the smaller exponent is shifted to the larger one.
__device__ __forceinline__ void acc_add(Acc &a, const WV &t) {
  uint32_t x[LA];
#pragma unroll
  for (int i = 0; i < LA; i++) x[i] = t.m.w[i + 1];
  const int32_t et = t.e + 32;
  const bool az = acc_is_zero(a);
  const int d = az ? 256 : et - a.e;  // > 0: the accumulator moves
  if (d > 0) {
    acc_sar(a, d);
    a.e = et;
  } else if (d < 0) {
    // logical right shift of the term by -d
    const int n = -d;
    if (n >= 224) {
#pragma unroll
      for (int i = 0; i < LA; i++) x[i] = 0u;
    } else {
      const bool s4 = (n & 128) != 0, s2 = (n & 64) != 0, s1 = (n & 32) != 0;
#pragma unroll
      for (int i = 0; i < LA; i++) x[i] = s4 ? (i + 4 < LA ? x[i + 4] : 0u) : x[i];
#pragma unroll
      for (int i = 0; i < LA; i++) x[i] = s2 ? (i + 2 < LA ? x[i + 2] : 0u) : x[i];
#pragma unroll
      for (int i = 0; i < LA; i++) x[i] = s1 ? (i + 1 < LA ? x[i + 1] : 0u) : x[i];
      const int b = n & 31;
#pragma unroll
      for (int i = 0; i < LA - 1; i++) x[i] = __funnelshift_r(x[i], x[i + 1], b);
      x[LA - 1] >>= b;
    }
  }
  acc_add_raw(a, x, t.s ? 0xffffffffu : 0u);
  acc_headroom(a);
}

// a += b for two accumulators.
__device__ __forceinline__ void acc_add_acc(Acc &a, Acc b) {
  if (acc_is_zero(b)) return;
  if (acc_is_zero(a)) {
    a = b;
    return;
  }
  if (b.e > a.e) {
    acc_sar(a, b.e - a.e);
    a.e = b.e;
  } else if (a.e > b.e) {
    acc_sar(b, a.e - b.e);
  }
  acc_add_raw(a, b.w, 0u);
  acc_headroom(a);
}

// ---------------------------------------------------------------------------
// rounding an accumulator to a quad-double
// ---------------------------------------------------------------------------

__device__ __forceinline__ int clz224(const uint32_t m[LA]) {
  int z = 224;
#pragma unroll
  for (int i = 0; i < LA; i++)
    if (m[i]) z = (LA - 1 - i) * 32 + __clz(static_cast<int>(m[i]));
  return z;
}

// x0 + x1 + x2 + x3 = A 2^e up to 2^-211 relative: each part is the value
// left by the parts before it rounded to the nearest double (ties away from
// zero in magnitude), so |x_{i+1}| <= ulp(x_i) / 2.  Zero gives four +0.0.
__device__ __forceinline__ void acc_to_qd(const Acc &a, double out[4]) {
  uint32_t M[LA];
  uint32_t neg = static_cast<uint32_t>(static_cast<int32_t>(a.w[LA - 1]) >> 31);
  // magnitude: (A ^ neg) + (neg & 1)
  uint32_t y[LA];
#pragma unroll
  for (int i = 0; i < LA; i++) y[i] = a.w[i] ^ neg;
  asm("{\n\t"
      ".reg .u32 t;\n\t"
      "and.b32         t, %14, 1;\n\t"
      "add.cc.u32      t, t, 0xffffffff;\n\t"
      "addc.cc.u32     %0, %7, 0;\n\t"
      "addc.cc.u32     %1, %8, 0;\n\t"
      "addc.cc.u32     %2, %9, 0;\n\t"
      "addc.cc.u32     %3, %10, 0;\n\t"
      "addc.cc.u32     %4, %11, 0;\n\t"
      "addc.cc.u32     %5, %12, 0;\n\t"
      "addc.u32        %6, %13, 0;\n\t"
      "}"
      : "=&r"(M[0]), "=&r"(M[1]), "=&r"(M[2]), "=&r"(M[3]), "=&r"(M[4]), "=&r"(M[5]), "=&r"(M[6])
      : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(neg));
  uint32_t s = neg & kSignBit;
#pragma unroll
  for (int part = 0; part < 4; part++) {
    const int lz = clz224(M);
    if (lz == 224) {
      out[part] = 0.0;
      continue;
    }
    const int p = 223 - lz;  // leading bit
    if (p <= 52) {           // the rest is exact in one double
      const unsigned long long v = (static_cast<unsigned long long>(M[1]) << 32) | M[0];
      out[part] = wide::make_double(v << (52 - p), a.e - (52 - p), s);
#pragma unroll
      for (int i = 0; i < LA; i++) M[i] = 0u;
      continue;
    }
    const int sh = p - 52;  // bits below the 53 kept ones
    // top 53 bits and the rounding bit
    uint32_t t[LA];
#pragma unroll
    for (int i = 0; i < LA; i++) t[i] = M[i];
    {
      const bool s4 = (sh & 128) != 0, s2 = (sh & 64) != 0, s1 = (sh & 32) != 0;
#pragma unroll
      for (int i = 0; i < LA; i++) t[i] = s4 ? (i + 4 < LA ? t[i + 4] : 0u) : t[i];
#pragma unroll
      for (int i = 0; i < LA; i++) t[i] = s2 ? (i + 2 < LA ? t[i + 2] : 0u) : t[i];
#pragma unroll
      for (int i = 0; i < LA; i++) t[i] = s1 ? (i + 1 < LA ? t[i + 1] : 0u) : t[i];
    }
    const int b = sh & 31;
    const uint32_t t0 = __funnelshift_r(t[0], t[1], b), t1 = __funnelshift_r(t[1], t[2], b);
    const unsigned long long top = (static_cast<unsigned long long>(t1) << 32) | t0;  // < 2^53
    const int rb = sh - 1;  // rounding bit position
    uint32_t rword = 0u;
#pragma unroll
    for (int i = 0; i < LA; i++) rword = (rb >> 5) == i ? M[i] : rword;
    const uint32_t round = (rword >> (rb & 31)) & 1u;
    const unsigned long long q = top + round;  // <= 2^53
    if (q >> 53)
      out[part] = wide::make_double(q >> 1, a.e + sh + 1, s);
    else
      out[part] = wide::make_double(q, a.e + sh, s);
    // remainder: low = M mod 2^sh; rounded up: 2^sh - low with the sign flipped
    const uint32_t rm = round ? 0xffffffffu : 0u;
#pragma unroll
    for (int i = 0; i < LA; i++) y[i] = M[i] ^ rm;
    asm("{\n\t"
        ".reg .u32 t;\n\t"
        "and.b32         t, %14, 1;\n\t"
        "add.cc.u32      t, t, 0xffffffff;\n\t"
        "addc.cc.u32     %0, %7, 0;\n\t"
        "addc.cc.u32     %1, %8, 0;\n\t"
        "addc.cc.u32     %2, %9, 0;\n\t"
        "addc.cc.u32     %3, %10, 0;\n\t"
        "addc.cc.u32     %4, %11, 0;\n\t"
        "addc.cc.u32     %5, %12, 0;\n\t"
        "addc.u32        %6, %13, 0;\n\t"
        "}"
        : "=&r"(M[0]), "=&r"(M[1]), "=&r"(M[2]), "=&r"(M[3]), "=&r"(M[4]), "=&r"(M[5]), "=&r"(M[6])
        : "r"(y[0]), "r"(y[1]), "r"(y[2]), "r"(y[3]), "r"(y[4]), "r"(y[5]), "r"(y[6]), "r"(rm));
#pragma unroll
    for (int i = 0; i < LA; i++) {
      const int lo = 32 * i;
      const uint32_t mask = sh >= lo + 32 ? 0xffffffffu : sh <= lo ? 0u : ((1u << (sh - lo)) - 1u);
      M[i] &= mask;
    }
    s ^= round ? kSignBit : 0u;
  }
}

// The sum of NP doubles rounded to a normalised quad-double (exact to about
// 2^-218 of the largest part, then the rounding of acc_to_qd).
template <int NP>
__device__ __forceinline__ void parts_to_qd(const double x[NP], double out[4]) {
  const Comp c = comp_from_parts<NP>(x);
  Acc a = acc_zero();
  acc_add(a, WV{c.m, c.s, c.e});
  acc_to_qd(a, out);
}

}  // namespace qd
}  // namespace pe
