// Newton's method on top of the evaluation (the use the paper evaluates f and
// J for, Section 1: the corrector of a path tracker).  One step at P points:
// solve J(x) dx = -f(x) by LU decomposition with partial pivoting, then
// x <- x + dx.
//
// One warp per point.  The Jacobian the evaluator wrote ([N][n][P], point
// index fastest) is factored in place; in elimination step k the lanes take
// the columns j > k of the trailing rows (lane j, j + 32, ...), the pivot is
// found by a warp-wide arg-max, the multipliers are formed by the lanes that
// own their rows, and the back substitution reduces each row's dot product
// across the warp.  Arithmetic in the precision of the evaluation
// (complex double-double, or complex double).  Right-hand side and solution
// overwrite f.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cplx.cuh"
#include "dd.cuh"
#include "internal.h"

namespace pe {


template <class C>
__global__ void newton_lu(const NewtonParams p) {
  constexpr int KD = C::kDoubles;
  const int lane = threadIdx.x & 31;
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;  // one warp per point
  if (q >= p.P) return;  // warp-uniform
  const int n = p.n;
  const size_t P = static_cast<size_t>(p.P);
  auto Jel = [&](int i, int j) { return p.J + ((static_cast<size_t>(i) * n + j) * P + q) * KD; };
  auto Fel = [&](int i) { return p.f + (static_cast<size_t>(i) * P + q) * KD; };
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * P + q) * KD; };

  // residual norm; right-hand side b = -f
  double fnorm = 0.0;
  for (int i = lane; i < n; i += 32) {
    const C fi = C::load(Fel(i));
    fnorm = fmax(fnorm, fi.abs_hi());
    fi.neg().store(Fel(i));
  }
  for (int d = 16; d > 0; d >>= 1) fnorm = fmax(fnorm, __shfl_xor_sync(kAll, fnorm, d));
  __syncwarp();

  bool singular = false;
  for (int k = 0; k < n; k++) {
    // pivot: the row i >= k of largest |J[i][k]| (smallest index on ties)
    double best = -1.0;
    int piv = n;
    for (int i = k + lane; i < n; i += 32) {
      const double m = C::load(Jel(i, k)).abs_hi();
      if (m > best) {
        best = m;
        piv = i;
      }
    }
    for (int d = 16; d > 0; d >>= 1) {
      const double ob = __shfl_xor_sync(kAll, best, d);
      const int op = __shfl_xor_sync(kAll, piv, d);
      if (ob > best || (ob == best && op < piv)) {
        best = ob;
        piv = op;
      }
    }
    if (!(best > 0.0)) {  // warp-uniform: this point's matrix is singular
      singular = true;
      break;
    }
    if (piv != k) {
      for (int j = k + lane; j < n; j += 32) {
        const C a = C::load(Jel(k, j)), b = C::load(Jel(piv, j));
        b.store(Jel(k, j));
        a.store(Jel(piv, j));
      }
      if (lane == 0) {
        const C a = C::load(Fel(k)), b = C::load(Fel(piv));
        b.store(Fel(k));
        a.store(Fel(piv));
      }
      __syncwarp();
    }
    // multipliers l_i = J[i][k] / J[k][k] and the right-hand side, by the
    // lanes that own rows i > k
    const C inv = C::recip(C::load(Jel(k, k)));
    const C bk = C::load(Fel(k));
    for (int i = k + 1 + lane; i < n; i += 32) {
      const C l = C::mul(C::load(Jel(i, k)), inv);
      l.store(Jel(i, k));
      C::sub_mul(C::load(Fel(i)), l, bk).store(Fel(i));
    }
    __syncwarp();
    // trailing update: lanes over the columns j > k
    for (int j = k + 1 + lane; j < n; j += 32) {
      const C u = C::load(Jel(k, j));
      for (int i = k + 1; i < n; i++) C::sub_mul(C::load(Jel(i, j)), C::load(Jel(i, k)), u).store(Jel(i, j));
    }
    __syncwarp();
  }

  // back substitution, dx overwrites b; each row's dot product reduced across the warp
  double dxnorm = 0.0;
  if (!singular) {
    for (int i = n - 1; i >= 0; i--) {
      C s = C::zero();
      for (int j = i + 1 + lane; j < n; j += 32) s = C::sub_mul(s, C::load(Jel(i, j)), C::load(Fel(j)));
      for (int d = 16; d > 0; d >>= 1) s = C::add2(s, s.shfl_down(d));
      if (lane == 0) {
        const C xi = C::mul(C::add2(C::load(Fel(i)), s).finish(), C::recip(C::load(Jel(i, i))));
        xi.store(Fel(i));
        dxnorm = fmax(dxnorm, xi.abs_hi());
      }
      __syncwarp();
    }
    dxnorm = __shfl_sync(kAll, dxnorm, 0);
    // x <- x + dx
    for (int i = lane; i < n; i += 32) C::add2(C::load(Xel(i)), C::load(Fel(i))).finish().store(Xel(i));
  } else {
    for (int i = lane; i < n; i += 32) C::zero().store(Fel(i));
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
