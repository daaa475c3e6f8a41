// Per-precision arithmetic of the lane-pair kernels (kernels.cu, newton.cu).
//
// Lanes 2q and 2q+1 hold the real and the imaginary part of the values of
// point q.  A policy gives the type one lane holds (V), the full complex value
// both lanes load (Full), and the operations on them; mul_x and mul_split are
// complex products with the partner lane's part fetched by a shuffle.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "dd.cuh"

namespace pe {

constexpr unsigned kFull = 0xffffffffu;
constexpr unsigned long long kSign = 0x8000000000000000ULL;

// ---------------------------------------------------------------------------
// precision policies: one real component per lane
// ---------------------------------------------------------------------------

struct ArithDD {
  using V = dd;         // one component (real or imaginary) held by a lane
  using F = dd;         // accumulator of f
  static constexpr int kDoubles = 4;  // doubles per complex element
  struct Full {
    dd re, im;
  };

  __device__ static Full load_full(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    return Full{dd{a.x, a.y}, dd{b.x, b.y}};
  }
  __device__ static void store_full(double *p, const Full &x) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(x.re.h, x.re.l);
    reinterpret_cast<double2 *>(p)[1] = make_double2(x.im.h, x.im.l);
  }
  __device__ static Full load_coherent(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return Full{dd{a.x, a.y}, dd{b.x, b.y}};
  }
  __device__ static V load_comp_ro(const double *p, int c) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p) + c);
    return dd{a.x, a.y};
  }
  __device__ static V load_comp(const double *p, int c) {
    const double2 a = reinterpret_cast<const double2 *>(p)[c];
    return dd{a.x, a.y};
  }
  __device__ static void store_comp(double *p, int c, V v) {
    reinterpret_cast<double2 *>(p)[c] = make_double2(v.h, v.l);
  }
  __device__ static V zero() { return dd{0.0, 0.0}; }
  __device__ static V comp(const Full &x, int c) { return select(c == 0, x.re, x.im); }
  __device__ static V im_signed(const Full &x, unsigned long long m) { return negate_if(x.im, m); }
  __device__ static V neg_if(V x, unsigned long long m) { return negate_if(x, m); }
  __device__ static V sel(bool t, V a, V b) { return select(t, a, b); }
  __device__ static V partner(V x, unsigned pm) {
    return dd{__shfl_xor_sync(pm, x.h, 1), __shfl_xor_sync(pm, x.l, 1)};
  }
  __device__ static F f_merge(F a, F b) { return pe::add(a, b); }
  __device__ static F f_xor(F a, int d) { return shfl_xor(a, d); }
  __device__ static V dot(V a1, V b1, V a2, V b2) { return dot2(a1, b1, a2, b2); }
  __device__ static V dotn(V a1, V b1, V a2, V b2) { return dot2n(a1, b1, a2, b2); }
  __device__ static V add(V a, V b) { return pe::add(a, b); }
  __device__ static V mul_int(V x, double k) { return scale(x, k); }
  __device__ static V finish(V x) { return normalize(x); }
  __device__ static F f_zero() { return dd{0.0, 0.0}; }
  __device__ static F f_add(F a, V x) { return pe::add(a, x); }
  __device__ static V f_finish(F a) { return normalize(a); }
  __device__ static Full cmul(const Full &x, const Full &y) {
    return Full{dot2n(x.re, y.re, negate_if(x.im, kSign), y.im), dot2n(x.re, y.im, x.im, y.re)};
  }
  __device__ static double hi(V x) { return x.h; }
  __device__ static V mul_real(V a, V b) { return mul(a, b); }
  __device__ static V recip_real(V d) { return recip(d); }
};

struct ArithF64 {
  using V = double;
  using F = dd;  // compensated sum of f: (running sum, sum of rounding errors)
  static constexpr int kDoubles = 2;
  struct Full {
    double re, im;
  };

  __device__ static Full load_full(const double *p) {
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    return Full{a.x, a.y};
  }
  __device__ static void store_full(double *p, const Full &x) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(x.re, x.im);
  }
  __device__ static Full load_coherent(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    return Full{a.x, a.y};
  }
  __device__ static V load_comp_ro(const double *p, int c) { return __ldg(p + c); }
  __device__ static V load_comp(const double *p, int c) { return p[c]; }
  __device__ static void store_comp(double *p, int c, V v) { p[c] = v; }
  __device__ static V zero() { return 0.0; }
  __device__ static V comp(const Full &x, int c) { return select(c == 0, x.re, x.im); }
  __device__ static V im_signed(const Full &x, unsigned long long m) { return negate_if(x.im, m); }
  __device__ static V neg_if(V x, unsigned long long m) { return negate_if(x, m); }
  __device__ static V sel(bool t, V a, V b) { return select(t, a, b); }
  __device__ static V partner(V x, unsigned pm) { return __shfl_xor_sync(pm, x, 1); }
  __device__ static F f_merge(F a, F b) {  // (s1 + e1) + (s2 + e2) with the rounding error of s1 + s2 kept
    double s, e;
    two_sum(a.h, b.h, s, e);
    return dd{s, __dadd_rn(__dadd_rn(a.l, b.l), e)};
  }
  __device__ static F f_xor(F a, int d) { return shfl_xor(a, d); }
  __device__ static V dot(V a1, V b1, V a2, V b2) { return __fma_rn(a1, b1, __dmul_rn(a2, b2)); }
  __device__ static V dotn(V a1, V b1, V a2, V b2) { return dot(a1, b1, a2, b2); }
  __device__ static V add(V a, V b) { return __dadd_rn(a, b); }
  __device__ static V mul_int(V x, double k) { return __dmul_rn(x, k); }
  __device__ static V finish(V x) { return x; }
  __device__ static F f_zero() { return dd{0.0, 0.0}; }
  __device__ static F f_add(F a, V x) {
    double s, e;
    two_sum(a.h, x, s, e);
    return dd{s, __dadd_rn(a.l, e)};
  }
  __device__ static V f_finish(F a) { return __dadd_rn(a.h, a.l); }
  __device__ static Full cmul(const Full &x, const Full &y) {
    return Full{__fma_rn(x.re, y.re, -__dmul_rn(x.im, y.im)), __fma_rn(x.re, y.im, __dmul_rn(x.im, y.re))};
  }
  __device__ static double hi(V x) { return x; }
  __device__ static V mul_real(V a, V b) { return __dmul_rn(a, b); }
  __device__ static V recip_real(V d) { return __ddiv_rn(1.0, d); }
};

// y * X for y split across the lane pair (this lane holds component c) and X
// a full complex value loaded by both lanes:
//   re: X.re y.re - X.im y.im     im: X.re y.im + X.im y.re
// i.e. X.re * y_own + (sign * X.im) * y_partner with sign -1 on real lanes.
// Norm: renormalise the result (for a product that feeds another product).
// pm: the mask of the lane pair (the whole warp when every lane works on the
// same monomial; the pair's two lanes when groups of the warp may diverge).
template <class A, bool Norm>
__device__ __forceinline__ typename A::V mul_x(typename A::V y, const typename A::Full &X, unsigned long long sgn,
                                               unsigned pm) {
  const typename A::V yp = A::partner(y, pm);
  return Norm ? A::dotn(X.re, y, A::im_signed(X, sgn), yp) : A::dot(X.re, y, A::im_signed(X, sgn), yp);
}

// P * Q with both factors split across the lane pair:
//   re lane: P.re Q.re - P.im Q.im      im lane: P.im Q.re + P.re Q.im
template <class A, bool Norm = false>
__device__ __forceinline__ typename A::V mul_split(typename A::V P, typename A::V Q, int c, unsigned long long sgn,
                                                   unsigned pm) {
  const typename A::V Pp = A::partner(P, pm);
  const typename A::V Qp = A::partner(Q, pm);
  const bool re = (c == 0);
  return Norm ? A::dotn(P, A::sel(re, Q, Qp), A::neg_if(Pp, sgn), A::sel(re, Qp, Q))
              : A::dot(P, A::sel(re, Q, Qp), A::neg_if(Pp, sgn), A::sel(re, Qp, Q));
}

// 1 / z for z split over the lane pair: conj(z) / |z|^2.
template <class A>
__device__ __forceinline__ typename A::V recip_split(typename A::V z, int c, unsigned pm) {
  const typename A::V zp = A::partner(z, pm);
  const typename A::V n2 = A::dotn(z, z, zp, zp);  // |z|^2, the same on both lanes
  return A::mul_real(A::neg_if(z, c ? kSign : 0ULL), A::recip_real(n2));
}

}  // namespace pe
