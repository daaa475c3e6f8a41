// Newton's method on top of the evaluation (the use the paper evaluates f and
// J for, Section 1: the corrector of a path tracker).  One step at P points:
// solve J(x) dx = -f(x) by LU decomposition with partial pivoting, then
// x <- x + dx.
//
// One warp per point factors the Jacobian the evaluator wrote ([N][n][P],
// point index fastest) in place (lu.cuh).  Arithmetic in the precision of the
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


template <class C>
__global__ void newton_lu(const NewtonParams p) {
  const int lane = threadIdx.x & 31;
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;  // one warp per point
  if (q >= p.P) return;  // warp-uniform
  const int n = p.n;
  const PointView<C> v{p.J, p.f, n, static_cast<size_t>(p.P), q};
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * p.P + q) * C::kDoubles; };

  // residual norm; right-hand side b = -f
  double fnorm = 0.0;
  for (int i = lane; i < n; i += 32) {
    const C fi = C::load(v.bel(i));
    fnorm = fmax(fnorm, fi.abs_hi());
    fi.neg().store(v.bel(i));
  }
  for (int d = 16; d > 0; d >>= 1) fnorm = fmax(fnorm, __shfl_xor_sync(kAll, fnorm, d));
  __syncwarp();

  const bool singular = lu_solve<C>(v, lane);
  double dxnorm = 0.0;
  if (!singular) {
    // x <- x + dx
    for (int i = lane; i < n; i += 32) {
      const C dx = C::load(v.bel(i));
      dxnorm = fmax(dxnorm, dx.abs_hi());
      C::add2(C::load(Xel(i)), dx).finish().store(Xel(i));
    }
    for (int d = 16; d > 0; d >>= 1) dxnorm = fmax(dxnorm, __shfl_xor_sync(kAll, dxnorm, d));
  } else {
    for (int i = lane; i < n; i += 32) C::zero().store(v.bel(i));
  }
  if (lane == 0 && p.norms) {
    p.norms[q * 2] = fnorm;
    p.norms[q * 2 + 1] = singular ? nan("") : dxnorm;
  }
}

cudaError_t launch_newton(bool dd, const NewtonParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.n <= 0) return cudaSuccess;
  const int threads = 128;
  const int64_t blocks = (p.P * 32 + threads - 1) / threads;
  if (dd)
    newton_lu<CDD><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  else
    newton_lu<C64><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pe
