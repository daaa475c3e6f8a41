// Solution of one point's linear system J y = b by LU decomposition with
// partial pivoting, by a segment of a warp, in place: either in the
// structure-of-arrays layout the evaluator writes (J [n][n][P], b [n][P],
// point index fastest; PointView) or in a copy in shared memory (row-major
// [n][n] and [n]; SmemView), which turns the chains of dependent global loads
// and stores of the elimination into shared-memory accesses.  Used by the
// Newton step (newton.cu) and the path tracker (track.cu).
//
// In elimination step k the pivot is the row of largest |J[i][k]| (by the
// leading parts, compared squared; the smallest index on ties) found by a
// segment-wide arg-max, the multipliers are formed by the lanes that own their
// rows, and the lanes of the segment share the (n-k-1)^2 elements of the
// trailing update in row order; the back substitution goes by columns, the
// lanes taking x_i out of the rows above it.  (One thread per point, each
// running a whole elimination, was slower at every batch size measured, up
// to 16384 points of 14 variables: its dependent chains of loads and stores
// leave the SMs waiting.)
// On return J holds the factors (unit lower triangle below the diagonal,
// after the row exchanges) and b the solution y.
#pragma once

#include <cstdint>

#include "cplx.cuh"

namespace pe {

// Element accessors of one point q in the [.][P] layouts.
template <class C>
struct PointView {
  double *J, *b;
  int n;
  size_t P;
  int64_t q;
  __device__ double *Jel(int i, int j) const { return J + ((static_cast<size_t>(i) * n + j) * P + q) * C::kDoubles; }
  __device__ double *bel(int i) const { return b + (static_cast<size_t>(i) * P + q) * C::kDoubles; }
};

// One point's system in shared memory: A row-major [n][n], b [n].
template <class C>
struct SmemView {
  double *A, *b;
  int n;
  __device__ double *Jel(int i, int j) const { return A + (static_cast<size_t>(i) * n + j) * C::kDoubles; }
  __device__ double *bel(int i) const { return b + static_cast<size_t>(i) * C::kDoubles; }
};

// Bytes of shared memory one warp needs for an n x n system, and the largest
// such copy staged in shared memory: larger systems are solved in global
// memory, where more warps per SM hide the latency (n = 32 in double-double,
// 34 KiB per warp, ran slower staged than in place: 4 warps per SM).
template <class C>
__host__ __device__ constexpr size_t smem_lu_bytes(int n) {
  return static_cast<size_t>(n) * (n + 1) * C::kDoubles * sizeof(double);
}
constexpr size_t kSmemLuMax = 16 * 1024;
// Threads per block of the segment kernels: one warp, so that a batch of a
// few warps per SM spreads evenly over the 152 SMs (with 4-warp blocks, 1024
// points at 32 lanes made 256 blocks: 2 on most SMs, 1 on the rest).
constexpr int kLuBlock = 32;

// max(a, b) that keeps a NaN (fmax drops it): a norm taken over values one of
// which is NaN is NaN, so a path or a Newton step that produced a NaN (an
// overflow, inf - inf) cannot pass a tolerance test on the other entries.
__device__ __forceinline__ double nan_max(double a, double b) { return (a != a || b != b) ? a + b : fmax(a, b); }

// The lanes that work on one point: S consecutive lanes of a warp (S a power
// of two, 4 .. 32) and the mask of their segment.  A warp holds 32 / S points,
// so that a small system does not leave most lanes idle: on GB300 an FP64
// warp instruction occupies the FP64 pipe for the same 16 cycles whatever
// its active lanes.  Shuffles and barriers use the segment's mask, so the
// points of one warp may take different branches.
template <int S>
struct Lanes {
  static constexpr int size = S;
  int lane;       // 0 .. S-1
  unsigned mask;  // the segment's lanes
  __device__ static Lanes of_thread() {
    const int t = static_cast<int>(threadIdx.x & 31);
    const unsigned m = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << (t & ~(S - 1)));
    return Lanes{t & (S - 1), m};
  }
  __device__ double max(double v) const {
    for (int d = S / 2; d > 0; d >>= 1) v = nan_max(v, __shfl_xor_sync(mask, v, d));
    return v;
  }
  __device__ void sync() const { __syncwarp(mask); }
};

// Lanes per point for an n x n system.
__host__ __device__ constexpr int lanes_for(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : 32; }

// Returns true (uniform over the segment) when a pivot column is exactly
// zero; b is then left partly eliminated.
template <class C, class V, int S>
__device__ bool lu_solve(const V &v, const Lanes<S> g) {
  const int n = v.n, lane = g.lane;
  for (int k = 0; k < n; k++) {
    double best = -1.0;
    int piv = n;
    for (int i = k + lane; i < n; i += S) {
      const double m = C::load(v.Jel(i, k)).norm2_hi();  // the modulus squared: same order, no square root
      if (m > best) {
        best = m;
        piv = i;
      }
    }
    for (int d = S / 2; d > 0; d >>= 1) {
      const double ob = __shfl_xor_sync(g.mask, best, d);
      const int op = __shfl_xor_sync(g.mask, piv, d);
      if (ob > best || (ob == best && op < piv)) {
        best = ob;
        piv = op;
      }
    }
    if (!(best > 0.0)) return true;  // uniform over the segment
    if (piv != k) {
      for (int j = k + lane; j < n; j += S) {
        const C a = C::load(v.Jel(k, j)), c = C::load(v.Jel(piv, j));
        c.store(v.Jel(k, j));
        a.store(v.Jel(piv, j));
      }
      if (lane == 0) {
        const C a = C::load(v.bel(k)), c = C::load(v.bel(piv));
        c.store(v.bel(k));
        a.store(v.bel(piv));
      }
      g.sync();
    }
    // multipliers l_i = J[i][k] / J[k][k] and the right-hand side
    const C inv = C::recip(C::load(v.Jel(k, k)));
    const C bk = C::load(v.bel(k));
    for (int i = k + 1 + lane; i < n; i += S) {
      const C l = C::mul(C::load(v.Jel(i, k)), inv);
      l.store(v.Jel(i, k));
      C::sub_mul(C::load(v.bel(i)), l, bk).store(v.bel(i));
    }
    g.sync();
    // trailing update: the lanes over the w x w elements (i, j > k) in row
    // order, so that all S lanes work until w^2 < S (lanes over the columns
    // alone would leave S - w idle at every step)
    const int w = n - k - 1;
    if (w > 0) {
      int i = k + 1 + lane / w, j = k + 1 + lane % w;
      const int di = S / w, dj = S % w;
      for (int e = lane; e < w * w; e += S) {
        C::sub_mul(C::load(v.Jel(i, j)), C::load(v.Jel(i, k)), C::load(v.Jel(k, j))).store(v.Jel(i, j));
        i += di;
        j += dj;
        if (j >= n) {
          j -= w;
          i++;
        }
      }
    }
    g.sync();
  }
  // back substitution, y overwrites b, by columns: x_i = y_i / U_ii (every
  // lane, which costs the FP64 pipe no more than one), then the lanes over
  // the rows r < i take x_i out of y_r
  for (int i = n - 1; i >= 0; i--) {
    const C xi = C::mul(C::load(v.bel(i)), C::recip(C::load(v.Jel(i, i))));
    g.sync();
    if (lane == 0) xi.store(v.bel(i));
    for (int r = lane; r < i; r += S) C::sub_mul(C::load(v.bel(r)), C::load(v.Jel(r, i)), xi).store(v.bel(r));
    g.sync();
  }
  return false;
}

}  // namespace pe

