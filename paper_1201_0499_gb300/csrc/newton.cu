// Newton's method on top of the evaluation (the use the paper evaluates f and
// J for, Section 1: the corrector of a path tracker).  One step at P points:
// solve J(x) dx = -f(x) by LU decomposition with partial pivoting, then
// x <- x + dx.
//
// One warp per point (or, for n <= 16, one thread per point) factors the
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

namespace pe {


template <class C, bool kSmem>
__global__ void newton_lu(const NewtonParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31;
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;  // one warp per point
  if (q >= p.P) return;  // warp-uniform
  const int n = p.n;
  const PointView<C> g{p.J, p.f, n, static_cast<size_t>(p.P), q};
  double *sm = reinterpret_cast<double *>(smem_raw) + (threadIdx.x >> 5) * (smem_lu_bytes<C>(n) / sizeof(double));
  const SmemView<C> sv{sm, sm + static_cast<size_t>(n) * n * C::kDoubles, n};
  auto bel = [&](int i) { return kSmem ? sv.bel(i) : g.bel(i); };
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * p.P + q) * C::kDoubles; };

  // residual norm; right-hand side b = -f
  double fnorm = 0.0;
  for (int i = lane; i < n; i += 32) {
    const C fi = C::load(g.bel(i));
    fnorm = fmax(fnorm, fi.abs_hi());
    fi.neg().store(bel(i));
  }
  for (int d = 16; d > 0; d >>= 1) fnorm = fmax(fnorm, __shfl_xor_sync(kAll, fnorm, d));
  if (kSmem)
    for (int e = lane; e < n * n; e += 32) C::load(g.Jel(e / n, e % n)).store(sv.Jel(e / n, e % n));
  __syncwarp();

  const bool singular = kSmem ? lu_solve<C>(sv, lane) : lu_solve<C>(g, lane);
  if (kSmem)  // the factors back to J
    for (int e = lane; e < n * n; e += 32) C::load(sv.Jel(e / n, e % n)).store(g.Jel(e / n, e % n));
  double dxnorm = 0.0;
  if (!singular) {
    // x <- x + dx; dx to f
    for (int i = lane; i < n; i += 32) {
      const C dx = C::load(bel(i));
      dxnorm = fmax(dxnorm, dx.abs_hi());
      dx.store(g.bel(i));
      C::add2(C::load(Xel(i)), dx).finish().store(Xel(i));
    }
    for (int d = 16; d > 0; d >>= 1) dxnorm = fmax(dxnorm, __shfl_xor_sync(kAll, dxnorm, d));
  } else {
    for (int i = lane; i < n; i += 32) C::zero().store(g.bel(i));
  }
  if (lane == 0 && p.norms) {
    p.norms[q * 2] = fnorm;
    p.norms[q * 2 + 1] = singular ? nan("") : dxnorm;
  }
}

// One thread per point (n <= kThreadLuMaxN).
template <class C>
__global__ void newton_lu_thread(const NewtonParams p) {
  const int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (q >= p.P) return;
  const int n = p.n;
  const PointView<C> g{p.J, p.f, n, static_cast<size_t>(p.P), q};
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * p.P + q) * C::kDoubles; };
  double fnorm = 0.0;
  for (int i = 0; i < n; i++) {
    const C fi = C::load(g.bel(i));
    fnorm = fmax(fnorm, fi.abs_hi());
    fi.neg().store(g.bel(i));
  }
  const bool singular = lu_solve_thread<C>(g);
  double dxnorm = 0.0;
  for (int i = 0; i < n; i++) {
    if (singular) {
      C::zero().store(g.bel(i));
    } else {
      const C dx = C::load(g.bel(i));
      dxnorm = fmax(dxnorm, dx.abs_hi());
      C::add2(C::load(Xel(i)), dx).finish().store(Xel(i));
    }
  }
  if (p.norms) {
    p.norms[q * 2] = fnorm;
    p.norms[q * 2 + 1] = singular ? nan("") : dxnorm;
  }
}

template <class C>
cudaError_t launch_newton_t(const NewtonParams &p, cudaStream_t s) {
  if (thread_lu(p.n, p.P)) {
    const int threads = 32;
    newton_lu_thread<C><<<static_cast<unsigned>((p.P + threads - 1) / threads), threads, 0, s>>>(p);
    return cudaGetLastError();
  }
  const size_t per_warp = smem_lu_bytes<C>(p.n);
  if (per_warp > kSmemLuMax) {
    const int threads = 128;
    const int64_t blocks = (p.P * 32 + threads - 1) / threads;
    newton_lu<C, false><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
    return cudaGetLastError();
  }
  const int warps = kSmemLuWarps;
  const size_t bytes = per_warp * warps;
  if (bytes > 48 * 1024) {
    const cudaError_t e =
        cudaFuncSetAttribute(newton_lu<C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
  }
  const int64_t blocks = (p.P + warps - 1) / warps;
  newton_lu<C, true><<<static_cast<unsigned>(blocks), warps * 32, bytes, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_newton(bool dd, const NewtonParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.n <= 0) return cudaSuccess;
  return dd ? launch_newton_t<CDD>(p, s) : launch_newton_t<C64>(p, s);
}

}  // namespace pe
