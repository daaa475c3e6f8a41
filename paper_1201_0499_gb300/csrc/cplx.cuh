// Complex numbers held whole by one thread (both parts), in double-double
// (CDD) and in double (C64): the arithmetic of the one-thread-per-item
// kernels (Newton solve, path tracker, the paper's three-kernel evaluation).
#pragma once

#include <cuda_runtime.h>

#include <cmath>

#include "dd.cuh"

namespace pe {
constexpr unsigned kAll = 0xffffffffu;

// complex double-double, both parts in one thread
struct CDD {
  static constexpr int kDoubles = 4;
  dd re, im;
  __device__ static CDD load(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    const double2 b = reinterpret_cast<const double2 *>(p)[1];
    return CDD{dd{a.x, a.y}, dd{b.x, b.y}};
  }
  __device__ void store(double *p) const {
    reinterpret_cast<double2 *>(p)[0] = make_double2(re.h, re.l);
    reinterpret_cast<double2 *>(p)[1] = make_double2(im.h, im.l);
  }
  __device__ static CDD zero() { return CDD{dd{0.0, 0.0}, dd{0.0, 0.0}}; }
  __device__ static CDD make(double re, double im) { return CDD{dd{re, 0.0}, dd{im, 0.0}}; }
  // x * k for a double k, renormalised
  __device__ static CDD scale(const CDD &x, double k) {
    return CDD{normalize(pe::scale(x.re, k)), normalize(pe::scale(x.im, k))};
  }
  __device__ static CDD sub(const CDD &a, const CDD &b) {
    return CDD{normalize(add(a.re, negate_if(b.re, 0x8000000000000000ULL))),
               normalize(add(a.im, negate_if(b.im, 0x8000000000000000ULL)))};
  }
  __device__ double abs_hi() const { return sqrt(re.h * re.h + im.h * im.h); }
  __device__ double norm2_hi() const { return __fma_rn(re.h, re.h, __dmul_rn(im.h, im.h)); }
  __device__ CDD neg() const { return CDD{negate_if(re, 0x8000000000000000ULL), negate_if(im, 0x8000000000000000ULL)}; }
  // x * y, renormalised
  __device__ static CDD mul(const CDD &x, const CDD &y) {
    return CDD{dot2n(x.re, y.re, negate_if(x.im, 0x8000000000000000ULL), y.im), dot2n(x.re, y.im, x.im, y.re)};
  }
  // a - x * y, renormalised
  __device__ static CDD sub_mul(const CDD &a, const CDD &x, const CDD &y) {
    const dd pr = dot2(x.re, y.re, negate_if(x.im, 0x8000000000000000ULL), y.im);
    const dd pi = dot2(x.re, y.im, x.im, y.re);
    return CDD{normalize(add(a.re, negate_if(pr, 0x8000000000000000ULL))),
               normalize(add(a.im, negate_if(pi, 0x8000000000000000ULL)))};
  }
  __device__ static CDD add2(const CDD &a, const CDD &b) { return CDD{add(a.re, b.re), add(a.im, b.im)}; }
  __device__ CDD finish() const { return CDD{normalize(re), normalize(im)}; }
  // 1 / z = conj(z) / |z|^2
  __device__ static CDD recip(const CDD &z) {
    const dd n2 = dot2n(z.re, z.re, z.im, z.im);
    const dd r = pe::recip(n2);
    return CDD{pe::mul(z.re, r), pe::mul(negate_if(z.im, 0x8000000000000000ULL), r)};
  }
  __device__ CDD shfl_xor(unsigned mask, int d) const {
    return CDD{dd{__shfl_xor_sync(mask, re.h, d), __shfl_xor_sync(mask, re.l, d)},
               dd{__shfl_xor_sync(mask, im.h, d), __shfl_xor_sync(mask, im.l, d)}};
  }
};

// complex double
struct C64 {
  static constexpr int kDoubles = 2;
  double re, im;
  __device__ static C64 load(const double *p) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0];
    return C64{a.x, a.y};
  }
  __device__ void store(double *p) const { reinterpret_cast<double2 *>(p)[0] = make_double2(re, im); }
  __device__ static C64 zero() { return C64{0.0, 0.0}; }
  __device__ static C64 make(double re, double im) { return C64{re, im}; }
  __device__ static C64 scale(const C64 &x, double k) { return C64{__dmul_rn(x.re, k), __dmul_rn(x.im, k)}; }
  __device__ static C64 sub(const C64 &a, const C64 &b) { return C64{__dsub_rn(a.re, b.re), __dsub_rn(a.im, b.im)}; }
  __device__ double abs_hi() const { return sqrt(re * re + im * im); }
  __device__ double norm2_hi() const { return __fma_rn(re, re, __dmul_rn(im, im)); }
  __device__ C64 neg() const { return C64{-re, -im}; }
  __device__ static C64 mul(const C64 &x, const C64 &y) {
    return C64{__fma_rn(x.re, y.re, -__dmul_rn(x.im, y.im)), __fma_rn(x.re, y.im, __dmul_rn(x.im, y.re))};
  }
  __device__ static C64 sub_mul(const C64 &a, const C64 &x, const C64 &y) {
    const C64 p = mul(x, y);
    return C64{__dsub_rn(a.re, p.re), __dsub_rn(a.im, p.im)};
  }
  __device__ static C64 add2(const C64 &a, const C64 &b) { return C64{__dadd_rn(a.re, b.re), __dadd_rn(a.im, b.im)}; }
  __device__ C64 finish() const { return *this; }
  __device__ static C64 recip(const C64 &z) {
    const double r = __ddiv_rn(1.0, __fma_rn(z.re, z.re, __dmul_rn(z.im, z.im)));
    return C64{__dmul_rn(z.re, r), -__dmul_rn(z.im, r)};
  }
  __device__ C64 shfl_xor(unsigned mask, int d) const {
    return C64{__shfl_xor_sync(mask, re, d), __shfl_xor_sync(mask, im, d)};
  }
};


// Conversions between the two (double-double to double keeps the leading
// parts, the nearest doubles of a renormalised value).
template <class L, class C>
__device__ __forceinline__ L convert(const C &x);
template <>
__device__ __forceinline__ CDD convert<CDD, CDD>(const CDD &x) { return x; }
template <>
__device__ __forceinline__ C64 convert<C64, C64>(const C64 &x) { return x; }
template <>
__device__ __forceinline__ C64 convert<C64, CDD>(const CDD &x) { return C64{x.re.h, x.im.h}; }
template <>
__device__ __forceinline__ CDD convert<CDD, C64>(const C64 &x) { return CDD{dd{x.re, 0.0}, dd{x.im, 0.0}}; }

}  // namespace pe

