// Kernels for the evaluation of a sparse polynomial system and its Jacobian
// (Verschelde & Yoffe, Sections 3.1-3.3), written for sm_103a.
//
// GB300 design (the paper's Tesla C2050 three-kernel design is prior art):
//
//  * The FP64 pipe is the bound: every value is a complex double-double (or
//    a complex double) and a double-precision instruction costs a warp 16 SM
//    cycles, so the kernels are laid out to issue as few of them as possible
//    and to keep at least one warp on every SM sub-partition.
//  * One warp evaluates one polynomial p of one system at a tile of 16
//    points.  Lanes 2q and 2q+1 hold the real and the imaginary part of every
//    value of point q, so a complex product is one double-double dot product
//    of length two per lane (13 FP64 instructions) plus shuffles with the
//    partner lane.  Every lane of the warp works on the same monomial: the
//    positions, exponents and coefficients are warp-uniform loads and
//    monomials of different k cause no divergence.
//  * Stage 1 (Section 3.1): the powers x_i^2 .. x_i^(d-1) are computed once
//    per point by a small kernel into a table in global memory (L2
//    resident); the common factor of a monomial is read from it.  The
//    coefficient is folded into the common factor, G = c prod x^(a-1).
//  * Stage 2 (Section 3.2): the forward products G x_{i_1} ... x_{i_j} are
//    kept in shared memory (one slot per variable per lane) and the backward
//    product Q in registers; d/dx_{i_j} of the term is a_j G prod_{l != j}
//    x_{i_l}.  A monomial with k variables costs #(a >= 2) + 3k - 3 complex
//    products instead of the paper's 6k - 5.
//  * Stage 3 (Section 3.3): the warp adds its terms straight into f (in
//    registers) and into the row J[p, :] of its points (read-modify-write in
//    the output array, which only this warp touches).  Only the nm(k+1) real
//    terms are added -- no zero padding -- in a fixed order, so results are
//    deterministic.  The row is renormalised once at the end.
//  * Work distribution: a persistent grid; each warp takes (polynomial,
//    tile) items from an atomic counter, most expensive first.
#include <cuda_runtime.h>

#include <cstdint>

#include "arith.cuh"
#include "dd.cuh"
#include "internal.h"
#include "items.cuh"

namespace pe {

template <class A>
__device__ __forceinline__ void accumulate(double *p, int c, bool valid, typename A::V d) {
  const typename A::V acc = A::add(A::load_comp(p, c), d);
  if (valid) A::store_comp(p, c, acc);
}

// One work item: polynomial gp (global index) of system s at the points of
// `tile`.  smem: this warp's prefix-product slots, [slot][lane].
template <class A>
__device__ void process_item(const MainParams &kp, const Item &it, typename A::V *smem, int lane) {
  const int gp = it.gp, tile = it.tile, s = it.s, P = it.P;
  using V = typename A::V;
  using Full = typename A::Full;
  constexpr int KD = A::kDoubles;
  const SysDesc sd = kp.sys[s];
  const int n = sd.n;
  const int q = tile * kPointsPerWarp + (lane >> 1);
  const bool valid = q < P;
  const int qc = valid ? q : P - 1;  // lanes past the end compute on the last point and store nothing
  const int c = lane & 1;
  const unsigned long long sgn = c ? 0ULL : kSign;
  const size_t Pz = static_cast<size_t>(P);
  const int pl = gp - sd.poly0;
  const double *X = kp.points + static_cast<size_t>(sd.pt_off) * KD;
  const double *Tb = kp.table + static_cast<size_t>(sd.tab_off) * KD;
  double *Jrow = it.J_base + (static_cast<size_t>(sd.J_off) + static_cast<size_t>(pl) * n * Pz) * KD;

  auto xel = [&](int v) { return X + (static_cast<size_t>(v) * Pz + qc) * KD; };
  auto tel = [&](int e, int v) { return Tb + ((static_cast<size_t>(e - 2) * n + v) * Pz + qc) * KD; };
  auto jel = [&](int v) { return Jrow + (static_cast<size_t>(v) * Pz + qc) * KD; };

  if (valid)
    for (int v = 0; v < n; v++) A::store_comp(jel(v), c, A::zero());

  typename A::F f = A::f_zero();
  const int t0 = it.t0, t1 = it.t1;
  for (int t = t0; t < t1; t++) {
    const int vb = kp.mono_ptr[t];
    const int k = kp.mono_ptr[t + 1] - vb;
    V G = A::load_comp_ro(kp.coef + static_cast<size_t>(t) * KD, c);
    if (k == 0) {  // constant term
      f = A::f_add(f, G);
      continue;
    }
    const uint32_t *vw = kp.var + vb;
    int step = 0;  // products since the last renormalisation (kChainRenorm)
    auto chain = [&](V y, const Full &X) {
      if (++step == kChainRenorm) {
        step = 0;
        return mul_x<A, true>(y, X, sgn, kFull);
      }
      return mul_x<A, false>(y, X, sgn, kFull);
    };
    // Stage 1: G = c * prod_{a_j >= 2} x_{i_j}^(a_j - 1)
    for (int j = 0; j < k; j++) {
      const uint32_t w = __ldg(vw + j);
      const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
      if (a >= 2) G = chain(G, A::load_full(a == 2 ? xel(v) : tel(a - 1, v)));
    }
    // Stage 2, forward: slot j <- G x_{i_1} ... x_{i_j}, j = 0 .. k-2
    V Pc = G;
    for (int j = 0; j < k - 1; j++) {
      smem[j * 32 + lane] = Pc;
      const int v = static_cast<int>(__ldg(vw + j) & 0xffffu);
      Pc = chain(Pc, A::load_full(xel(v)));
    }
    // value c x^a = Pc x_{i_k}; derivative by x_{i_k} = a_k Pc
    const uint32_t wl = __ldg(vw + k - 1);
    const int vl = static_cast<int>(wl & 0xffffu), al = static_cast<int>(wl >> 16);
    const Full xl = A::load_full(xel(vl));
    f = A::f_add(f, mul_x<A, false>(Pc, xl, sgn, kFull));
    accumulate<A>(jel(vl), c, valid, al == 1 ? Pc : A::mul_int(Pc, int_as_double(al)));
    // Stage 2, backward: Q = x_{i_{j+2}} ... x_{i_k}; derivative by x_{i_{j+1}} = a_{j+1} slot_j Q
    V Q = A::comp(xl, c);
    step = 0;
    for (int j = k - 2; j >= 0; j--) {
      const uint32_t w = __ldg(vw + j);
      const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
      const V D = mul_split<A>(smem[j * 32 + lane], Q, c, sgn, kFull);
      accumulate<A>(jel(v), c, valid, a == 1 ? D : A::mul_int(D, int_as_double(a)));
      if (j > 0) Q = chain(Q, A::load_full(xel(v)));
    }
  }
  if (valid) {
    A::store_comp(it.f_base + (static_cast<size_t>(sd.f_off) + static_cast<size_t>(pl) * Pz + q) * KD, c,
                  A::f_finish(f));
    for (int v = 0; v < n; v++) {
      double *p = jel(v);
      A::store_comp(p, c, A::finish(A::load_comp(p, c)));
    }
  }
}

// The same with G monomial groups per warp (G = 2, 4, 8, 16): each group of
// 32 / G lanes holds the 16 / G points of the tile (lanes 2q, 2q+1 of the
// group: point q) and the G groups take monomials t0 + g, t0 + g + G, ... of
// the polynomial, so that a
// call with few points keeps every lane busy (the "threads per monomial"
// choice: 32 / G lanes per monomial).  Groups of one round may have monomials
// of different k and diverge, so the partner shuffles use the pair's mask.
// Each group keeps its derivative terms in its slots and the groups add them
// into the row J[p, :] one after another (two monomials of a round may share
// a variable); f is summed per group and across the groups at the end.
template <class A, int G>
__device__ void process_item_groups(const MainParams &kp, const Item &it, typename A::V *smem, int lane) {
  constexpr int GL = 32 / G;                     // lanes per group
  constexpr int QP = kPointsPerWarp / G;         // points per tile
  const int gp = it.gp, tile = it.tile, s = it.s, P = it.P;
  using V = typename A::V;
  using Full = typename A::Full;
  constexpr int KD = A::kDoubles;
  const SysDesc sd = kp.sys[s];
  const int n = sd.n;
  const int g = lane / GL;
  const int q = tile * QP + ((lane % GL) >> 1);
  const bool valid = q < P;
  const int qc = valid ? q : P - 1;
  const int c = lane & 1;
  const unsigned long long sgn = c ? 0ULL : kSign;
  const unsigned pm = 3u << (lane & 30);
  const size_t Pz = static_cast<size_t>(P);
  const int pl = gp - sd.poly0;
  const double *X = kp.points + static_cast<size_t>(sd.pt_off) * KD;
  const double *Tb = kp.table + static_cast<size_t>(sd.tab_off) * KD;
  double *Jrow = it.J_base + (static_cast<size_t>(sd.J_off) + static_cast<size_t>(pl) * n * Pz) * KD;

  auto xel = [&](int v) { return X + (static_cast<size_t>(v) * Pz + qc) * KD; };
  auto tel = [&](int e, int v) { return Tb + ((static_cast<size_t>(e - 2) * n + v) * Pz + qc) * KD; };
  auto jel = [&](int v) { return Jrow + (static_cast<size_t>(v) * Pz + qc) * KD; };

  if (valid && g == 0)
    for (int v = 0; v < n; v++) A::store_comp(jel(v), c, A::zero());
  __syncwarp();

  typename A::F f = A::f_zero();
  const int t0 = it.t0, t1 = it.t1;
  for (int base = t0; base < t1; base += G) {
    const int t = base + g;
    const bool has = t < t1;  // uniform over the group
    int k = 0;
    const uint32_t *vw = nullptr;
    if (has) {
      const int vb = kp.mono_ptr[t];
      k = kp.mono_ptr[t + 1] - vb;
      vw = kp.var + vb;
      V Gv = A::load_comp_ro(kp.coef + static_cast<size_t>(t) * KD, c);
      if (k == 0) {
        f = A::f_add(f, Gv);
      } else {
        int step = 0;
        auto chain = [&](V y, const Full &Xf) {
          if (++step == kChainRenorm) {
            step = 0;
            return mul_x<A, true>(y, Xf, sgn, pm);
          }
          return mul_x<A, false>(y, Xf, sgn, pm);
        };
        for (int j = 0; j < k; j++) {
          const uint32_t w = __ldg(vw + j);
          const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
          if (a >= 2) Gv = chain(Gv, A::load_full(a == 2 ? xel(v) : tel(a - 1, v)));
        }
        V Pc = Gv;
        for (int j = 0; j < k - 1; j++) {
          smem[j * 32 + lane] = Pc;
          const int v = static_cast<int>(__ldg(vw + j) & 0xffffu);
          Pc = chain(Pc, A::load_full(xel(v)));
        }
        const uint32_t wl = __ldg(vw + k - 1);
        const int vl = static_cast<int>(wl & 0xffffu), al = static_cast<int>(wl >> 16);
        const Full xl = A::load_full(xel(vl));
        f = A::f_add(f, mul_x<A, false>(Pc, xl, sgn, pm));
        // derivative terms into the slots: slot j <- term of x_{i_{j+1}}
        V Q = A::comp(xl, c);
        step = 0;
        for (int j = k - 2; j >= 0; j--) {
          const int a = static_cast<int>(__ldg(vw + j) >> 16);
          const V D = mul_split<A>(smem[j * 32 + lane], Q, c, sgn, pm);
          smem[j * 32 + lane] = a == 1 ? D : A::mul_int(D, int_as_double(a));
          if (j > 0) Q = chain(Q, A::load_full(xel(static_cast<int>(__ldg(vw + j) & 0xffffu))));
        }
        smem[(k - 1) * 32 + lane] = al == 1 ? Pc : A::mul_int(Pc, int_as_double(al));
      }
    }
    __syncwarp();
    for (int r = 0; r < G; r++) {  // the groups' terms into J, one group at a time
      if (g == r && k > 0)
        for (int j = 0; j < k; j++) accumulate<A>(jel(static_cast<int>(__ldg(vw + j) & 0xffffu)), c, valid, smem[j * 32 + lane]);
      __syncwarp();
    }
  }
  for (int d = GL; d < 32; d <<= 1) f = A::f_merge(f, A::f_xor(f, d));
  if (valid && g == 0) {
    A::store_comp(it.f_base + (static_cast<size_t>(sd.f_off) + static_cast<size_t>(pl) * Pz + q) * KD, c,
                  A::f_finish(f));
    for (int v = 0; v < n; v++) {
      double *p = jel(v);
      A::store_comp(p, c, A::finish(A::load_comp(p, c)));
    }
  }
}

template <class A, int G>
__global__ void main_kernel(const MainParams kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  typename A::V *smem = reinterpret_cast<typename A::V *>(smem_raw) + static_cast<size_t>(warp) * kp.kslots * 32;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(kp.counter, 1u);
    item = __shfl_sync(kFull, item, 0);
    if (static_cast<int64_t>(item) >= kp.n_items) break;
    Item it;
    if (!decode_item(kp, item, lane, it)) continue;
    if constexpr (G == 1)
      process_item<A>(kp, it, smem, lane);
    else
      process_item_groups<A, G>(kp, it, smem, lane);
  }
}

// Stage 1 table: x^e for e = 2 .. emax-1 of every (system, variable, point).
template <class A>
__global__ void powers_kernel(const PowerParams pp) {
  constexpr int KD = A::kDoubles;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < pp.total; idx += stride) {
    int n, emax, P;
    int64_t local, pt_off, tab_off;
    if (pp.single_P >= 0) {
      n = pp.single_n;
      emax = pp.single_emax;
      P = pp.single_P;
      local = idx;
      pt_off = 0;
      tab_off = 0;
    } else {
      int lo = 0, hi = pp.count;  // find s with prefix[s] <= idx < prefix[s+1]
      while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (pp.prefix[mid] <= idx) lo = mid; else hi = mid;
      }
      const SysDesc sd = pp.sys[lo];
      n = sd.n;
      emax = sd.emax;
      P = sd.P;
      local = idx - pp.prefix[lo];
      pt_off = sd.pt_off;
      tab_off = sd.tab_off;
    }
    const int64_t v = local / P, q = local - v * P;
    const typename A::Full x = A::load_full(pp.points + (pt_off + v * P + q) * KD);
    auto entry = [&](int e) { return pp.table + (tab_off + (static_cast<int64_t>(e - 2) * n + v) * P + q) * KD; };
    // x^e = x^(e - h) * x^h with h = floor(e/2): one product per entry as in
    // a running product, but a rounding chain of depth O(log e), not O(e).
    for (int e = 2; e < emax; e++) {
      const int h = e >> 1, g = e - h;
      const typename A::Full lo = h == 1 ? x : A::load_coherent(entry(h));
      const typename A::Full hi = g == 1 ? x : A::load_coherent(entry(g));
      A::store_full(entry(e), A::cmul(hi, lo));
    }
  }
}

// out[i] += sum of the chunk partials, renormalised (one component per thread).
template <class A>
__global__ void combine_kernel(double *out, const double *scratch, int64_t comps, int64_t stride, int chunks) {
  constexpr int CD = A::kDoubles / 2;  // doubles per component
  const int64_t step = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < comps; i += step) {
    typename A::V acc = A::load_comp(out + i * CD, 0);
    for (int c = 1; c < chunks; c++) acc = A::add(acc, A::load_comp(scratch + (c - 1) * stride + i * CD, 0));
    A::store_comp(out + i * CD, 0, A::finish(acc));
  }
}

cudaError_t launch_combine(bool dd, double *out_f, double *out_J, const double *scratch_f, const double *scratch_J,
                           int64_t f_doubles, int64_t J_doubles, int chunks, cudaStream_t s) {
  if (chunks <= 1) return cudaSuccess;
  const int threads = 256;
  for (int pass = 0; pass < 2; pass++) {
    double *out = pass ? out_J : out_f;
    const double *scr = pass ? scratch_J : scratch_f;
    const int64_t doubles = pass ? J_doubles : f_doubles;
    const int64_t comps = dd ? doubles / 2 : doubles;
    if (comps <= 0) continue;
    int64_t blocks = (comps + threads - 1) / threads;
    if (blocks > kSms * 64) blocks = kSms * 64;
    if (dd)
      combine_kernel<ArithDD><<<static_cast<unsigned>(blocks), threads, 0, s>>>(out, scr, comps, doubles, chunks);
    else
      combine_kernel<ArithF64><<<static_cast<unsigned>(blocks), threads, 0, s>>>(out, scr, comps, doubles, chunks);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_powers(bool dd, const PowerParams &p, cudaStream_t s) {
  if (p.total <= 0) return cudaSuccess;
  const int threads = 256;
  int64_t blocks = (p.total + threads - 1) / threads;
  if (blocks > kSms * 64) blocks = kSms * 64;
  if (dd)
    powers_kernel<ArithDD><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  else
    powers_kernel<ArithF64><<<static_cast<unsigned>(blocks), threads, 0, s>>>(p);
  return cudaGetLastError();
}

// Batch handles: each item carries its own number of monomial groups (the
// last, partial tile of a system spreads its few points over the warp).
template <class A>
__global__ void main_kernel_batch(const MainParams kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  typename A::V *smem = reinterpret_cast<typename A::V *>(smem_raw) + static_cast<size_t>(warp) * kp.kslots * 32;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(kp.counter, 1u);
    item = __shfl_sync(kFull, item, 0);
    if (static_cast<int64_t>(item) >= kp.n_items) break;
    Item it;
    if (!decode_item(kp, item, lane, it)) continue;
    switch (it.groups) {
      case 2: process_item_groups<A, 2>(kp, it, smem, lane); break;
      case 4: process_item_groups<A, 4>(kp, it, smem, lane); break;
      case 8: process_item_groups<A, 8>(kp, it, smem, lane); break;
      case 16: process_item_groups<A, 16>(kp, it, smem, lane); break;
      default: process_item<A>(kp, it, smem, lane); break;
    }
  }
}

template <class A>
cudaError_t prepare_main_t(int v) {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(main_kernel<A, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) ||
      (e = cudaFuncSetAttribute(main_kernel<A, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) ||
      (e = cudaFuncSetAttribute(main_kernel<A, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) ||
      (e = cudaFuncSetAttribute(main_kernel<A, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) ||
      (e = cudaFuncSetAttribute(main_kernel<A, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)) ||
      (e = cudaFuncSetAttribute(main_kernel_batch<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, v)))
    return e;
  return cudaSuccess;
}

cudaError_t prepare_main(bool dd, size_t smem_bytes) {
  // Every handle launches with at most the device's opt-in limit; setting the
  // attribute to that limit once keeps it valid for all handles.
  const int v = static_cast<int>(smem_bytes);
  return dd ? prepare_main_t<ArithDD>(v) : prepare_main_t<ArithF64>(v);
}

cudaError_t main_occupancy(bool dd, bool batch, int warps_per_block, size_t smem_bytes, int *blocks_per_sm) {
  const int t = warps_per_block * 32;
  if (batch)
    return dd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel_batch<ArithDD>, t, smem_bytes)
              : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel_batch<ArithF64>, t, smem_bytes);
  return dd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel<ArithDD, 1>, t, smem_bytes)
            : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_kernel<ArithF64, 1>, t, smem_bytes);
}

template <class A>
cudaError_t launch_main_t(const MainParams &p, int warps_per_block, size_t smem_bytes, int grid, cudaStream_t s) {
  const dim3 b(warps_per_block * 32);
  if (p.single_P < 0) {
    main_kernel_batch<A><<<grid, b, smem_bytes, s>>>(p);
    return cudaGetLastError();
  }
  switch (p.groups) {
    case 1: main_kernel<A, 1><<<grid, b, smem_bytes, s>>>(p); break;
    case 2: main_kernel<A, 2><<<grid, b, smem_bytes, s>>>(p); break;
    case 4: main_kernel<A, 4><<<grid, b, smem_bytes, s>>>(p); break;
    case 8: main_kernel<A, 8><<<grid, b, smem_bytes, s>>>(p); break;
    case 16: main_kernel<A, 16><<<grid, b, smem_bytes, s>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_main(bool dd, const MainParams &p, int warps_per_block, size_t smem_bytes, int grid,
                        cudaStream_t s) {
  if (p.n_items <= 0) return cudaSuccess;
  return dd ? launch_main_t<ArithDD>(p, warps_per_block, smem_bytes, grid, s)
            : launch_main_t<ArithF64>(p, warps_per_block, smem_bytes, grid, s);
}

// ---------------------------------------------------------------------------
// FP64 issue-rate probe: independent FMA chains on every SM.
// ---------------------------------------------------------------------------

__global__ void fp64_probe_kernel(double *out, long long *cycles, int iters) {
  double acc[8];
#pragma unroll
  for (int i = 0; i < 8; i++) acc[i] = threadIdx.x * 1e-3 + i;
  const double a = 1.0000001, b = 1e-9;
  const long long c0 = clock64();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int i = 0; i < 8; i++) acc[i] = __fma_rn(acc[i], a, b);
  }
  const long long c1 = clock64();
  double sum = 0.0;
#pragma unroll
  for (int i = 0; i < 8; i++) sum += acc[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = sum;
  if (threadIdx.x == 0) cycles[blockIdx.x] = c1 - c0;
}

cudaError_t fp64_peak_probe(cudaStream_t s, double *fma_per_s, double *sm_clock_mhz) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  const int blocks = sms * 4, threads = 256, iters = 1000;
  double *out = nullptr;
  long long *cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  long long *hc = nullptr;
  if ((e = cudaMalloc(&out, sizeof(double) * blocks * threads)) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&cyc, sizeof(long long) * blocks)) != cudaSuccess) goto done;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) goto done;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) goto done;
  fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, cyc, 64);  // warm-up
  cudaEventRecord(e0, s);
  fp64_probe_kernel<<<blocks, threads, 0, s>>>(out, cyc, iters);
  cudaEventRecord(e1, s);
  if ((e = cudaEventSynchronize(e1)) != cudaSuccess) goto done;
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  {
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    hc = new long long[blocks];
    if ((e = cudaMemcpy(hc, cyc, sizeof(long long) * blocks, cudaMemcpyDeviceToHost)) != cudaSuccess) goto done;
    long long mc = 0;
    for (int i = 0; i < blocks; i++) mc = hc[i] > mc ? hc[i] : mc;
    const double ops = static_cast<double>(blocks) * threads * iters * 8.0;
    if (fma_per_s) *fma_per_s = ops / (ms * 1e-3);
    if (sm_clock_mhz) *sm_clock_mhz = static_cast<double>(mc) / (ms * 1e-3) / 1e6;
  }
done:
  delete[] hc;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (cyc) cudaFree(cyc);
  return e;
}

}  // namespace pe
