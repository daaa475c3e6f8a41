// Predictor-corrector path tracking on top of the evaluation: the use the
// paper evaluates f and J for (Section 1: Newton's method as the corrector of
// a path tracker solving polynomial systems by homotopy continuation).
//
// Homotopy (total degree, with the "gamma trick"):
//   H(x, t) = gamma (1 - t) G(x) + t F(x),   G_i(x) = x_i^(d_i) - 1,
// d_i the degree of polynomial i of the target system F, gamma a random
// complex constant.  At t = 0 the solutions are the products of roots of
// unity; each one is followed to t = 1.
//
// One step kernel per iteration, one warp per path, after the evaluator has
// written F(x) and J_F(x) for every path at its current point x.  A path is a
// small state machine:
//   CORRECT  Newton step on H(., t1) = 0; accepted when
//            max|dx| <= corr_tol max(1, max|x|), rejected after max_corr
//            steps or when the steps stop shrinking (x back to the last
//            accepted point, h halved; below h_min the path fails);
//   PREDICT  Euler step along the tangent: H_x v = -H_t, with
//            H_t = F - gamma G; x += (t1 - t) v with t1 = min(t + h, 1);
//   END      at t = 1, Newton on F until max|dx| <= end_tol max(1, max|x|)
//            (success) or max_end steps (endpoint not converged).
// After succ_grow accepted steps in a row the step size doubles (up to h_max).
// Paths whose max|x| exceeds x_big are marked diverged.
//
// Mixed precision (double-double tracking with `mixed` set): the homotopy,
// the right-hand sides and the points stay in double-double, the linear
// systems are solved in double from the leading parts of H_x (in shared
// memory or in the tracker's double scratch).  Each corrector step is then a step of iterative
// refinement, whose error falls by about u cond(H_x) (u = 2^-53) per step, and
// the step kernel runs about a tenth of the FP64 instructions of a
// double-double LU -- on GB300, whose FP64 pipe issues a warp instruction in
// 16 cycles whatever the active lanes, that is most of a tracker iteration.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cplx.cuh"
#include "internal.h"
#include "lu.cuh"

namespace pe {

namespace {

template <class C>
__device__ __forceinline__ C cpow(C x, int e) {  // x^e for e >= 0, by squaring
  C r = C::make(1.0, 0.0);
  while (e > 0) {
    if (e & 1) r = C::mul(r, x);
    e >>= 1;
    if (e) x = C::mul(x, x);
  }
  return r;
}


}  // namespace

// One step of path q by the S lanes of grp.  C: the tracker's arithmetic; L:
// that of the linear solve (C, or C64 for mixed precision).  kSmem: the
// system is staged in the segment's shared memory; else it is formed in the
// evaluator's J and f (L == C) or in the scratch p.JL, p.bL (L != C).
template <class C, class L, bool kSmem, class G>
__device__ void track_path(const TrackParams &p, int64_t q, const G grp, double *sm) {
  TrackState s = p.st[q];
  if (s.status != kPathRunning) return;  // uniform over the group
  const int n = p.n, lane = grp.lane;
  const size_t P = static_cast<size_t>(p.P);
  const PointView<C> g{p.J, p.f, n, P, q};
  const SmemView<L> sv{sm, sm + static_cast<size_t>(n) * n * L::kDoubles, n};
  // the in-place system: the evaluator's arrays, or the double scratch
  constexpr bool kScratch = !kSmem && sizeof(L) != sizeof(C);
  const PointView<L> gl{kScratch ? p.JL : p.J, kScratch ? p.bL : p.f, n, P, q};
  auto Ael = [&](int i, int j) { return kSmem ? sv.Jel(i, j) : gl.Jel(i, j); };
  auto bel = [&](int i) { return kSmem ? sv.bel(i) : gl.bel(i); };
  auto Xel = [&](double *base, int i) { return base + (static_cast<size_t>(i) * P + q) * C::kDoubles; };
  const C gamma = C::make(p.gre, p.gim);

  // the homotopy at (x, tt): matrix H_x, right-hand side
  const bool predict = s.phase == kPhasePredict;
  const double tt = predict ? s.t : (s.phase == kPhaseEnd ? 1.0 : s.t1);
  const C a = C::scale(gamma, 1.0 - tt);  // gamma (1 - t)
  const L al = convert<L>(a);
  for (int e = lane, i = lane / n, j = lane % n; e < n * n; e += G::size) {  // the n^2 entries over the lanes
    L v = L::scale(convert<L>(C::load(g.Jel(i, j))), tt);
    if (j == i) {
      const L xi = convert<L>(C::load(Xel(p.x, i)));
      const int d = p.deg[i];
      v = L::add2(v, L::mul(al, L::scale(cpow(xi, d - 1), static_cast<double>(d)))).finish();
    }
    v.store(Ael(i, j));
    i += G::size / n;
    j += G::size % n;
    if (j >= n) {
      j -= n;
      i++;
    }
  }
  for (int i = lane; i < n; i += G::size) {
    const C xi = C::load(Xel(p.x, i));
    const C Gi = C::sub(cpow(xi, p.deg[i]), C::make(1.0, 0.0));
    const C F = C::load(g.bel(i));
    C rhs;
    if (predict)  // -H_t = gamma G - F
      rhs = C::sub(C::mul(gamma, Gi), F);
    else  // -H = -(a G + t F)
      rhs = C::add2(C::mul(a, Gi), C::scale(F, tt)).finish().neg();
    convert<L>(rhs).store(bel(i));
  }
  grp.sync();

  bool singular;
  if constexpr (kSmem)
    singular = lu_solve<L>(sv, grp);
  else
    singular = lu_solve<L>(gl, grp);

  auto restore = [&]() {  // x <- last accepted point
    for (int i = lane; i < n; i += G::size) C::load(Xel(p.xs, i)).store(Xel(p.x, i));
  };
  auto reject = [&]() {
    restore();
    s.h *= 0.5;
    s.succ = 0;
    s.iter = 0;
    s.phase = kPhasePredict;
    if (s.h < p.h_min) s.status = kPathFailed;
  };

  if (singular) {
    if (s.phase == kPhaseEnd)
      s.status = kPathEndNotConverged;
    else
      reject();
  } else if (predict) {
    s.t1 = fmin(s.t + s.h, 1.0);
    const double dt = s.t1 - s.t;
    for (int i = lane; i < n; i += G::size)
      C::add2(C::load(Xel(p.x, i)), C::scale(convert<C>(L::load(bel(i))), dt)).finish().store(Xel(p.x, i));
    s.phase = kPhaseCorrect;
    s.iter = 0;
    s.dprev = INFINITY;
  } else {
    double dxn = 0.0, xn = 0.0;
    for (int i = lane; i < n; i += G::size) {
      const C dx = convert<C>(L::load(bel(i)));
      const C x1 = C::add2(C::load(Xel(p.x, i)), dx).finish();
      x1.store(Xel(p.x, i));
      dxn = nan_max(dxn, dx.abs_hi());
      xn = nan_max(xn, x1.abs_hi());
    }
    dxn = grp.max(dxn);
    xn = grp.max(xn);
    s.iter++;
    const double scale = fmax(1.0, xn);
    if (!(xn <= p.x_big) || !(dxn == dxn) || isinf(xn)) {  // beyond x_big, or not finite
      s.status = kPathDiverged;
    } else if (s.phase == kPhaseEnd) {
      if (dxn <= p.end_tol * scale)
        s.status = kPathSuccess;
      else if (s.iter >= p.max_end)
        s.status = kPathEndNotConverged;
    } else if (dxn <= p.corr_tol * scale) {  // accept
      s.t = s.t1;
      for (int i = lane; i < n; i += G::size) C::load(Xel(p.x, i)).store(Xel(p.xs, i));
      if (++s.succ >= p.succ_grow) {
        s.h = fmin(2.0 * s.h, p.h_max);
        s.succ = 0;
      }
      s.iter = 0;
      s.phase = s.t >= 1.0 ? kPhaseEnd : kPhasePredict;
    } else if (s.iter >= p.max_corr || (s.iter >= 2 && dxn > s.dprev)) {
      reject();
    } else {
      s.dprev = dxn;
    }
  }
  grp.sync();
  if (lane == 0) {
    p.st[q] = s;
    if (s.status == kPathRunning) atomicAdd(p.active, 1u);
  }
}

// S lanes per path (32 / S paths per warp).
template <class C, class L, bool kSmem, int S>
__global__ void track_step(const TrackParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t q = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) / S;
  if (q >= p.P) return;  // uniform over the segment
  double *sm = reinterpret_cast<double *>(smem_raw) + (threadIdx.x / S) * (smem_lu_bytes<L>(p.n) / sizeof(double));
  track_path<C, L, kSmem>(p, q, Lanes<S>::of_thread(), sm);
}

__global__ void track_init(const TrackParams p, double h_init, int words) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < p.P; q += stride) {
    TrackState s;
    s.t = 0.0;
    s.t1 = 0.0;  // first: correct the start point at t = 0
    s.h = h_init;
    s.dprev = INFINITY;
    s.phase = kPhaseCorrect;
    s.iter = 0;
    s.succ = 0;
    s.status = kPathRunning;
    p.st[q] = s;
    for (int i = 0; i < p.n; i++)
      for (int w = 0; w < words; w++) {
        const size_t o = (static_cast<size_t>(i) * p.P + q) * words + w;
        p.xs[o] = p.x[o];
      }
  }
}

__global__ void track_finish(const TrackState *st, int64_t P, double *t, int32_t *status) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t q = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; q < P; q += stride) {
    if (t) t[q] = st[q].t;
    if (status) status[q] = st[q].status;
  }
}

// Start solutions of G(x) = 0: path r = first + j has the mixed-radix digits
// k_i of r (radices d_0, d_1, ...) and x_i = exp(2 pi i k_i / d_i).
__global__ void start_points(int32_t n, const int32_t *deg, int64_t first, int64_t P, double *x, int words) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < P; j += stride) {
    int64_t r = first + j;
    for (int i = 0; i < n; i++) {
      const int64_t d = deg[i];
      const int64_t k = r % d;
      r /= d;
      double sn, cs;
      sincospi(2.0 * static_cast<double>(k) / static_cast<double>(d), &sn, &cs);
      double *e = x + (static_cast<size_t>(i) * P + j) * words;
      for (int w = 0; w < words; w++) e[w] = 0.0;
      e[0] = cs;
      e[words / 2] = sn;
    }
  }
}

// Conversions between complex double-double [.][4] and double [.][2], and
// gathers/scatters of whole paths (all n variables of a point).
__global__ void narrow_points(const double *dd, double *c64, int64_t count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count; e += stride) {
    c64[2 * e] = dd[4 * e];
    c64[2 * e + 1] = dd[4 * e + 2];
  }
}

__global__ void widen_points(const double *c64, double *dd, int64_t count) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < count; e += stride) {
    dd[4 * e] = c64[2 * e];
    dd[4 * e + 1] = 0.0;
    dd[4 * e + 2] = c64[2 * e + 1];
    dd[4 * e + 3] = 0.0;
  }
}

// dst[i][j] = src[i][idx[j]] (gather) or dst[i][idx[j]] = src[i][j] (scatter),
// for i < n, j < m; entries of `words` doubles.
__global__ void move_paths(const double *src, int64_t P_src, double *dst, int64_t P_dst, const int64_t *idx,
                           int64_t m, int32_t n, int words, bool scatter) {
  const int64_t total = m * n;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t e = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < total; e += stride) {
    const int64_t i = e / m, j = e - i * m;
    const int64_t from = scatter ? j : idx[j], to = scatter ? idx[j] : j;
    const double *a = src + (i * P_src + from) * words;
    double *b = dst + (i * P_dst + to) * words;
    for (int w = 0; w < words; w++) b[w] = a[w];
  }
}

__global__ void scatter_status(const int32_t *src, int32_t *dst, const int64_t *idx, int64_t m) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < m; j += stride) dst[idx[j]] = src[j];
}

namespace {
constexpr int kTrackWarpsLatency = kSms * 8;

// Lanes per path: as many as the system needs (lanes_for), doubled while
// the batch would leave fewer than 8 warps per SM: the step is a chain of
// dependent FP64 operations, latency bound in small batches (late in a run,
// when most paths have ended), and the LU's element-wise updates spread
// over the extra lanes.
int track_lanes(int n, int64_t P) {
  int S = lanes_for(n);
  while (S < 32 && P * S < static_cast<int64_t>(kTrackWarpsLatency) * 32) S *= 2;
  return S;
}

unsigned grid_for(int64_t work, int threads) {
  int64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > kSms * 32) b = kSms * 32;
  return static_cast<unsigned>(b);
}
}  // namespace

cudaError_t launch_track_init(bool dd, const TrackParams &p, double h_init, cudaStream_t s) {
  if (p.P <= 0) return cudaSuccess;
  track_init<<<grid_for(p.P, 256), 256, 0, s>>>(p, h_init, dd ? 4 : 2);
  return cudaGetLastError();
}

template <class C, class L, int S>
cudaError_t launch_track_segments(const TrackParams &p, cudaStream_t s) {
  const int64_t blocks = (p.P * S + kLuBlock - 1) / kLuBlock;
  const size_t per_path = smem_lu_bytes<L>(p.n);
  if (per_path > kSmemLuMax) {
    track_step<C, L, false, S><<<static_cast<unsigned>(blocks), kLuBlock, 0, s>>>(p);
    return cudaGetLastError();
  }
  const size_t bytes = per_path * (kLuBlock / S);
  if (bytes > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(track_step<C, L, true, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(bytes));
    if (e != cudaSuccess) return e;
  }
  track_step<C, L, true, S><<<static_cast<unsigned>(blocks), kLuBlock, bytes, s>>>(p);
  return cudaGetLastError();
}

template <class C, class L>
cudaError_t launch_track_step_t(const TrackParams &p, cudaStream_t s) {
  switch (track_lanes(p.n, p.P)) {
    case 4: return launch_track_segments<C, L, 4>(p, s);
    case 8: return launch_track_segments<C, L, 8>(p, s);
    case 16: return launch_track_segments<C, L, 16>(p, s);
    default: return launch_track_segments<C, L, 32>(p, s);
  }
}

cudaError_t launch_track_step(bool dd, const TrackParams &p, cudaStream_t s) {
  if (p.P <= 0) return cudaSuccess;
  if (!dd) return launch_track_step_t<C64, C64>(p, s);
  return p.mixed ? launch_track_step_t<CDD, C64>(p, s) : launch_track_step_t<CDD, CDD>(p, s);
}

cudaError_t launch_track_finish(const TrackState *st, int64_t P, double *t, int32_t *status, cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  track_finish<<<grid_for(P, 256), 256, 0, s>>>(st, P, t, status);
  return cudaGetLastError();
}

cudaError_t launch_start_points(bool dd, int32_t n, const int32_t *deg, int64_t first, int64_t P, double *x,
                                cudaStream_t s) {
  if (P <= 0) return cudaSuccess;
  start_points<<<grid_for(P, 128), 128, 0, s>>>(n, deg, first, P, x, dd ? 4 : 2);
  return cudaGetLastError();
}

cudaError_t launch_narrow_points(const double *dd, double *c64, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  narrow_points<<<grid_for(count, 256), 256, 0, s>>>(dd, c64, count);
  return cudaGetLastError();
}

cudaError_t launch_widen_points(const double *c64, double *dd, int64_t count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  widen_points<<<grid_for(count, 256), 256, 0, s>>>(c64, dd, count);
  return cudaGetLastError();
}

cudaError_t launch_move_paths(const double *src, int64_t P_src, double *dst, int64_t P_dst, const int64_t *idx,
                              int64_t m, int32_t n, int words, bool scatter, cudaStream_t s) {
  if (m <= 0 || n <= 0) return cudaSuccess;
  move_paths<<<grid_for(m * n, 256), 256, 0, s>>>(src, P_src, dst, P_dst, idx, m, n, words, scatter);
  return cudaGetLastError();
}

cudaError_t launch_scatter_status(const int32_t *src, int32_t *dst, const int64_t *idx, int64_t m, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  scatter_status<<<grid_for(m, 256), 256, 0, s>>>(src, dst, idx, m);
  return cudaGetLastError();
}

}  // namespace pe
