// Newton's method on top of the evaluation (the use the paper evaluates f and
// J for, Section 1: the corrector of a path tracker).  One step at P points:
// solve J(x) dx = -f(x) by LU decomposition with partial pivoting, then
// x <- x + dx.
//
// One lane pair per point (lanes 2q and 2q+1: real and imaginary parts), in
// the precision of the evaluation (double-double, or double).  The Jacobian
// the evaluator wrote ([N][n][P], point index fastest) is factored in place:
// every load and store of a warp covers 16 consecutive points, coalesced.
// Right-hand side and solution overwrite f.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "arith.cuh"
#include "internal.h"

namespace pe {

template <class A>
__global__ void newton_solve(const NewtonParams p) {
  using V = typename A::V;
  constexpr int KD = A::kDoubles;
  const int lane = threadIdx.x & 31;
  const int64_t warp = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  if (warp * kPointsPerWarp >= p.P) return;  // the whole warp is past the end
  const int64_t q = warp * kPointsPerWarp + (lane >> 1);
  const bool valid = q < p.P;
  const int64_t qc = valid ? q : p.P - 1;  // lanes past the end compute on the last point and store nothing
  const int c = lane & 1;
  const unsigned long long sgn = c ? 0ULL : kSign;
  const unsigned long long neg = kSign;
  const int n = p.n;
  const size_t P = static_cast<size_t>(p.P);
  auto Jel = [&](int i, int j) { return p.J + ((static_cast<size_t>(i) * n + j) * P + qc) * KD; };
  auto Fel = [&](int i) { return p.f + (static_cast<size_t>(i) * P + qc) * KD; };
  auto Xel = [&](int i) { return p.x + (static_cast<size_t>(i) * P + qc) * KD; };
  auto mag = [&](V z) {  // |z| of the pair's complex value, from the high words
    const double a = A::hi(z), b = A::hi(A::partner(z));
    return sqrt(a * a + b * b);
  };

  // residual norm; right-hand side b = -f
  double fnorm = 0.0;
  for (int i = 0; i < n; i++) {
    const V fi = A::load_comp(Fel(i), c);
    fnorm = fmax(fnorm, mag(fi));
    if (valid) A::store_comp(Fel(i), c, A::neg_if(fi, neg));
  }

  bool singular = false;
  for (int k = 0; k < n; k++) {
    int piv = k;
    double best = -1.0;
    for (int i = k; i < n; i++) {
      const double m = mag(A::load_comp(Jel(i, k), c));
      if (m > best) {
        best = m;
        piv = i;
      }
    }
    // a zero pivot column: this point's matrix is singular; the pair carries
    // on with a zero multiplier (no branch around the shuffles below)
    const bool zero_pivot = !(best > 0.0);
    singular = singular || zero_pivot;
    if (piv != k && valid) {
      for (int j = k; j < n; j++) {
        const V a = A::load_comp(Jel(k, j), c), b = A::load_comp(Jel(piv, j), c);
        A::store_comp(Jel(k, j), c, b);
        A::store_comp(Jel(piv, j), c, a);
      }
      const V a = A::load_comp(Fel(k), c), b = A::load_comp(Fel(piv), c);
      A::store_comp(Fel(k), c, b);
      A::store_comp(Fel(piv), c, a);
    }
    V inv = recip_split<A>(A::load_comp(Jel(k, k), c), c);
    if (zero_pivot) inv = A::zero();
    const V bk = A::load_comp(Fel(k), c);
    for (int i = k + 1; i < n; i++) {
      const V l = mul_split<A, true>(A::load_comp(Jel(i, k), c), inv, c, sgn);  // multiplier l_ik
      if (valid) A::store_comp(Jel(i, k), c, l);
      for (int j = k + 1; j < n; j++) {
        const V t = mul_split<A>(l, A::load_comp(Jel(k, j), c), c, sgn);
        const V a = A::add(A::load_comp(Jel(i, j), c), A::neg_if(t, neg));
        if (valid) A::store_comp(Jel(i, j), c, A::finish(a));
      }
      const V b = A::add(A::load_comp(Fel(i), c), A::neg_if(mul_split<A>(l, bk, c, sgn), neg));
      if (valid) A::store_comp(Fel(i), c, A::finish(b));
    }
  }

  // back substitution: dx overwrites the right-hand side
  double dxnorm = 0.0;
  for (int i = n - 1; i >= 0; i--) {
    V s = A::load_comp(Fel(i), c);
    for (int j = i + 1; j < n; j++)
      s = A::add(s, A::neg_if(mul_split<A>(A::load_comp(Jel(i, j), c), A::load_comp(Fel(j), c), c, sgn), neg));
    V dx = mul_split<A, true>(A::finish(s), recip_split<A>(A::load_comp(Jel(i, i), c), c), c, sgn);
    if (singular) dx = A::zero();
    dxnorm = fmax(dxnorm, mag(dx));
    if (valid) A::store_comp(Fel(i), c, dx);
  }
  // x <- x + dx
  if (!singular) {
    for (int i = 0; i < n; i++) {
      const V x = A::add(A::load_comp(Xel(i), c), A::load_comp(Fel(i), c));
      if (valid) A::store_comp(Xel(i), c, A::finish(x));
    }
  }
  if (valid && p.norms) p.norms[q * 2 + c] = c == 0 ? fnorm : (singular ? nan("") : dxnorm);
}

cudaError_t launch_newton(bool dd, const NewtonParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.n <= 0) return cudaSuccess;
  const int64_t warps = (p.P + kPointsPerWarp - 1) / kPointsPerWarp;
  const int threads = 64;
  const int64_t blocks = (warps * 32 + threads - 1) / threads;
  if (dd)
    newton_solve<ArithDD><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  else
    newton_solve<ArithF64><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pe
