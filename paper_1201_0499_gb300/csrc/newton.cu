// Newton's method on top of the evaluation (the use the paper evaluates f and
// J for, Section 1: the corrector of a path tracker).  One step at P points:
// solve J(x) dx = -f(x) by LU decomposition with partial pivoting, then
// x <- x + dx.
//
// A segment of a warp per point (4 to 32 lanes as n needs) factors the
// Jacobian the evaluator wrote ([N][n][P], point index fastest) in place
// (lu.cuh).  Arithmetic in the precision of the
// evaluation (complex double-double, or complex double).  Right-hand side and
// solution overwrite f.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cplx.cuh"
#include "dd.cuh"
#include "internal.h"
#include "lu.cuh"
#include "wide8.cuh"

namespace pe {


template <class C, bool kSmem, int S>
__global__ void newton_lu(const NewtonParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / S;  // S lanes per point
  if (q >= p.P) return;  // uniform over the segment
  const Lanes<S> g = Lanes<S>::of_thread();
  const int lane = g.lane;
  const int n = p.n;
  const PointView<C> gv{p.J, p.f, n, static_cast<size_t>(p.P), q};
  double *sm = reinterpret_cast<double *>(smem_raw) + (threadIdx.x / S) * (smem_lu_bytes<C>(n) / sizeof(double));
  const SmemView<C> sv{sm, sm + static_cast<size_t>(n) * n * C::kDoubles, n};
  auto bel = [&](int i) { return kSmem ? sv.bel(i) : gv.bel(i); };
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * p.P + q) * C::kDoubles; };

  // residual norm; right-hand side b = -f
  double fnorm = 0.0;
  for (int i = lane; i < n; i += S) {
    const C fi = C::load(gv.bel(i));
    fnorm = nan_max(fnorm, fi.abs_hi());
    fi.neg().store(bel(i));
  }
  fnorm = g.max(fnorm);
  if (kSmem)
    for (int e = lane; e < n * n; e += S) C::load(gv.Jel(e / n, e % n)).store(sv.Jel(e / n, e % n));
  g.sync();

  const bool singular = kSmem ? lu_solve<C>(sv, g) : lu_solve<C>(gv, g);
  if (kSmem)  // the factors back to J
    for (int e = lane; e < n * n; e += S) C::load(sv.Jel(e / n, e % n)).store(gv.Jel(e / n, e % n));
  double dxnorm = 0.0;
  if (!singular) {
    // x <- x + dx; dx to f
    for (int i = lane; i < n; i += S) {
      const C dx = C::load(bel(i));
      dxnorm = nan_max(dxnorm, dx.abs_hi());
      dx.store(gv.bel(i));
      C::add2(C::load(Xel(i)), dx).finish().store(Xel(i));
    }
    dxnorm = g.max(dxnorm);
  } else {
    for (int i = lane; i < n; i += S) C::zero().store(gv.bel(i));
  }
  if (lane == 0 && p.norms) {
    p.norms[q * 2] = fnorm;
    p.norms[q * 2 + 1] = singular ? nan("") : dxnorm;
  }
}

template <class C, int S>
cudaError_t launch_newton_segments(const NewtonParams &p, cudaStream_t s) {
  const int64_t blocks = (p.P * S + kLuBlock - 1) / kLuBlock;
  const size_t per_point = smem_lu_bytes<C>(p.n);
  if (per_point > kSmemLuMax) {
    newton_lu<C, false, S><<<static_cast<unsigned>(blocks), kLuBlock, 0, s>>>(p);
    return cudaGetLastError();
  }
  const size_t bytes = per_point * (kLuBlock / S);
  if (bytes > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(newton_lu<C, true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
  }
  newton_lu<C, true, S><<<static_cast<unsigned>(blocks), kLuBlock, bytes, s>>>(p);
  return cudaGetLastError();
}

template <class C>
cudaError_t launch_newton_t(const NewtonParams &p, cudaStream_t s) {
  switch (lanes_for(p.n)) {
    case 4: return launch_newton_segments<C, 4>(p, s);
    case 8: return launch_newton_segments<C, 8>(p, s);
    case 16: return launch_newton_segments<C, 16>(p, s);
    default: return launch_newton_segments<C, 32>(p, s);
  }
}

// Newton step for quad-double handles: the residual f and the Jacobian J
// come from the quad-double evaluation ([.][P] of 8 doubles); the correction
// solves J dx = -f in double-double from their leading two parts per
// component (an iterative-refinement step: the error of x falls by about
// 2^-104 cond(J) per step, down to the quad-double floor), and x + dx is
// summed exactly on the integer pipe and rounded to a normalised quad-double.
// On return f holds dx (as a quad-double with two zero parts) and J the
// double-double factors in the leading parts.  The double-double system is
// staged in shared memory, or in the scratch p.Jdd, p.fdd when too large.
template <bool kSmem, int S>
__global__ void newton_qd(const NewtonParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / S;
  if (q >= p.P) return;  // uniform over the segment
  const Lanes<S> g = Lanes<S>::of_thread();
  const int lane = g.lane;
  const int n = p.n;
  const size_t P = static_cast<size_t>(p.P);
  double *sm = reinterpret_cast<double *>(smem_raw) + (threadIdx.x / S) * (smem_lu_bytes<CDD>(n) / sizeof(double));
  const SmemView<CDD> sv{sm, sm + static_cast<size_t>(n) * n * 4, n};
  const PointView<CDD> gv{p.Jdd, p.fdd, n, P, q};
  auto Ael = [&](int i, int j) { return kSmem ? sv.Jel(i, j) : gv.Jel(i, j); };
  auto bel = [&](int i) { return kSmem ? sv.bel(i) : gv.bel(i); };
  auto Jq = [&](int i, int j) { return p.J + ((static_cast<size_t>(i) * n + j) * P + q) * 8; };
  auto fq = [&](int i) { return p.f + (static_cast<size_t>(i) * P + q) * 8; };
  auto xq = [&](int i) { return p.x + (static_cast<size_t>(i) * P + q) * 8; };
  auto lead = [](const double *e) {  // the leading two parts of each component
    const double2 r = reinterpret_cast<const double2 *>(e)[0], m = reinterpret_cast<const double2 *>(e)[2];
    return CDD{dd{r.x, r.y}, dd{m.x, m.y}};
  };
  auto store_qd = [](double *e, const CDD &v) {
    reinterpret_cast<double2 *>(e)[0] = make_double2(v.re.h, v.re.l);
    reinterpret_cast<double2 *>(e)[1] = make_double2(0.0, 0.0);
    reinterpret_cast<double2 *>(e)[2] = make_double2(v.im.h, v.im.l);
    reinterpret_cast<double2 *>(e)[3] = make_double2(0.0, 0.0);
  };

  double fnorm = 0.0;
  for (int i = lane; i < n; i += S) {
    const CDD fi = lead(fq(i));
    fnorm = nan_max(fnorm, fi.abs_hi());
    fi.neg().store(bel(i));
  }
  fnorm = g.max(fnorm);
  for (int e = lane; e < n * n; e += S) lead(Jq(e / n, e % n)).store(Ael(e / n, e % n));
  g.sync();

  const bool singular = kSmem ? lu_solve<CDD>(sv, g) : lu_solve<CDD>(gv, g);
  for (int e = lane; e < n * n; e += S) store_qd(Jq(e / n, e % n), CDD::load(Ael(e / n, e % n)));
  double dxnorm = 0.0;
  for (int i = lane; i < n; i += S) {
    if (singular) {
      store_qd(fq(i), CDD::zero());
      continue;
    }
    const CDD dx = CDD::load(bel(i));
    dxnorm = nan_max(dxnorm, dx.abs_hi());
    double *x = xq(i);
    for (int c = 0; c < 2; c++) {  // x_c + dx_c, six parts summed exactly, rounded to four
      const dd d = c == 0 ? dx.re : dx.im;
      const double parts[6] = {x[4 * c], x[4 * c + 1], x[4 * c + 2], x[4 * c + 3], d.h, d.l};
      double out[4];
      qd::parts_to_qd<6>(parts, out);
      reinterpret_cast<double2 *>(x + 4 * c)[0] = make_double2(out[0], out[1]);
      reinterpret_cast<double2 *>(x + 4 * c)[1] = make_double2(out[2], out[3]);
    }
    store_qd(fq(i), dx);
  }
  dxnorm = g.max(dxnorm);
  if (lane == 0 && p.norms) {
    p.norms[q * 2] = fnorm;
    p.norms[q * 2 + 1] = singular ? nan("") : dxnorm;
  }
}

template <int S>
cudaError_t launch_newton_qd_segments(const NewtonParams &p, cudaStream_t s) {
  const int64_t blocks = (p.P * S + kLuBlock - 1) / kLuBlock;
  const size_t per_point = smem_lu_bytes<CDD>(p.n);
  if (per_point > kSmemLuMax) {
    if (!p.Jdd || !p.fdd) return cudaErrorInvalidValue;
    newton_qd<false, S><<<static_cast<unsigned>(blocks), kLuBlock, 0, s>>>(p);
    return cudaGetLastError();
  }
  const size_t bytes = per_point * (kLuBlock / S);
  if (bytes > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(newton_qd<true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
  }
  newton_qd<true, S><<<static_cast<unsigned>(blocks), kLuBlock, bytes, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_newton_qd(const NewtonParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.n <= 0) return cudaSuccess;
  switch (lanes_for(p.n)) {
    case 4: return launch_newton_qd_segments<4>(p, s);
    case 8: return launch_newton_qd_segments<8>(p, s);
    case 16: return launch_newton_qd_segments<16>(p, s);
    default: return launch_newton_qd_segments<32>(p, s);
  }
}

bool newton_qd_needs_scratch(int n) { return smem_lu_bytes<CDD>(n) > kSmemLuMax; }

cudaError_t launch_newton(bool dd, const NewtonParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.n <= 0) return cudaSuccess;
  return dd ? launch_newton_t<CDD>(p, s) : launch_newton_t<C64>(p, s);
}

}  // namespace pe
