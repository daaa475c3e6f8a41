// Kernels of the integer-pipe evaluation (precision PE_DD_INT): the same
// method and work decomposition as kernels.cu (Sections 3.1-3.3 of the
// paper), with every product in the 128-bit block floating point of
// wide.cuh and the sums into f and J in double-double on the FP64 pipe, so
// that the integer pipes carry the products and the FP64 pipe the sums.
//
//  * powers_wide: every point's variables converted to the block format and
//    their powers x^2 .. x^(d-1), in a table [e-1][n][P] of 48-byte entries
//    (entry e = 1 is x itself).
//  * main_wide: one warp per (polynomial, tile of 16 points); lanes 2q and
//    2q+1 hold the real and the imaginary part of point q.  Common factor
//    with the coefficient folded in, forward products in shared memory
//    ([slot][word][lane], conflict-free), value, backward running product,
//    derivatives; each term is converted to a double-double and added into f
//    (registers) or the row J[p, :] (read-modify-write in the output).
#include <cuda_runtime.h>

#include <cstdint>

#include "dd.cuh"
#include "internal.h"
#include "items.cuh"
#include "wide.cuh"

namespace pe {

using wide::WF;
using wide::WV;

constexpr int kWideWords = 12;  // 32-bit words per stored full value (48 bytes)
constexpr int kSlotWords = 5;   // words per lane in a prefix-product slot (4 limbs, sign | exponent)

__global__ void convert_coef_kernel(const double *coef_dd, uint32_t *coef_wide, int64_t M) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < M; t += stride) {
    const double *c = coef_dd + t * 4;
    wide::store_wf(coef_wide + t * kWideWords, wide::wf_from_cdd(c[0], c[1], c[2], c[3]));
  }
}

__global__ void powers_wide(const PowerParams pp) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  uint32_t *table = reinterpret_cast<uint32_t *>(pp.table);
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
      int lo = 0, hi = pp.count;
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
    const double *xp = pp.points + (pt_off + v * P + q) * 4;
    auto entry = [&](int e) { return table + (tab_off + (static_cast<int64_t>(e - 1) * n + v) * P + q) * kWideWords; };
    const WF x = wide::wf_from_cdd(xp[0], xp[1], xp[2], xp[3]);
    wide::store_wf(entry(1), x);
    for (int e = 2; e < emax; e++) {
      const int h = e >> 1, g = e - h;
      const WF a = h == 1 ? x : wide::load_wf_coherent(entry(h));
      const WF b = g == 1 ? x : wide::load_wf_coherent(entry(g));
      wide::store_wf(entry(e), wide::wf_mul(b, a));
    }
  }
}

__device__ __forceinline__ void store_slot(uint32_t *slots, int j, int lane, const WV &v) {
  uint32_t *b = slots + j * (kSlotWords * 32) + lane;
  b[0] = v.m.w0;
  b[32] = v.m.w1;
  b[64] = v.m.w2;
  b[96] = v.m.w3;
  b[128] = v.s | (static_cast<uint32_t>(v.e) & 0x7fffffffu);  // exponents fit in 31 bits
}

__device__ __forceinline__ WV load_slot(const uint32_t *slots, int j, int lane) {
  const uint32_t *b = slots + j * (kSlotWords * 32) + lane;
  const uint32_t se = b[128];
  return WV{wide::Mag{b[0], b[32], b[64], b[96]}, se & wide::kSignBit, static_cast<int32_t>(se << 1) >> 1};
}

__device__ __forceinline__ void accumulate_dd(double *p, int c, bool valid, dd x) {
  const double2 a = reinterpret_cast<const double2 *>(p)[c];
  const dd s = add(dd{a.x, a.y}, x);
  if (valid) reinterpret_cast<double2 *>(p)[c] = make_double2(s.h, s.l);
}

// One work item.  Pf: the table value of the next product and the J entry
// of the next derivative term are read one step ahead, so that their L2 (or
// DRAM) latency overlaps the current product's carry chains; this holds about
// 30 more registers per thread, which pays where shared memory already limits
// the resident warps (large k) and costs occupancy where it does not.
template <bool Pf>
__device__ void process_item_wide(const MainParams &kp, const Item &it, uint32_t *slots, int lane) {
  const int gp = it.gp, tile = it.tile, s = it.s, P = it.P;
  const SysDesc sd = kp.sys[s];
  const int n = sd.n;
  const int q = tile * kPointsPerWarp + (lane >> 1);
  const bool valid = q < P;
  const int qc = valid ? q : P - 1;
  const int c = lane & 1;
  const size_t Pz = static_cast<size_t>(P);
  const int pl = gp - sd.poly0;
  const uint32_t *Tb = reinterpret_cast<const uint32_t *>(kp.table) + static_cast<size_t>(sd.tab_off) * kWideWords;
  const uint32_t *coef = reinterpret_cast<const uint32_t *>(kp.coef);
  double *Jrow = it.J_base + (static_cast<size_t>(sd.J_off) + static_cast<size_t>(pl) * n * Pz) * 4;

  auto tel = [&](int e, int v) { return Tb + ((static_cast<size_t>(e - 1) * n + v) * Pz + qc) * kWideWords; };
  auto jel = [&](int v) { return Jrow + (static_cast<size_t>(v) * Pz + qc) * 4; };
  auto xw = [&](const uint32_t *vw, int j) { return wide::load_wf(tel(1, static_cast<int>(__ldg(vw + j) & 0xffffu))); };

  if (valid)
    for (int v = 0; v < n; v++) reinterpret_cast<double2 *>(jel(v))[c] = make_double2(0.0, 0.0);

  dd f{0.0, 0.0};
  const int t0 = it.t0, t1 = it.t1;
  for (int t = t0; t < t1; t++) {
    const int vb = kp.mono_ptr[t];
    const int k = kp.mono_ptr[t + 1] - vb;
    WV G = wide::component(wide::load_wf(coef + static_cast<size_t>(t) * kWideWords), c);
    if (k == 0) {
      f = add(f, wide::to_dd(G));
      continue;
    }
    const uint32_t *vw = kp.var + vb;
    // chain products: every second one normalised (see wide::mul_x)
    bool norm = false;
    auto chain = [&](const WV &y, const WF &X) {
      const WV r = norm ? wide::mul_x<true>(y, X, c) : wide::mul_x<false>(y, X, c);
      norm = !norm;
      return r;
    };
    // Stage 1: G = c * prod_{a_j >= 2} x_{i_j}^(a_j - 1)
    if constexpr (Pf) {
      int j = 0;
      uint32_t w = 0;
      for (; j < k; j++) {
        w = __ldg(vw + j);
        if ((w >> 16) >= 2) break;
      }
      WF xa;
      if (j < k) xa = wide::load_wf(tel(static_cast<int>(w >> 16) - 1, static_cast<int>(w & 0xffffu)));
      while (j < k) {
        const WF xc = xa;
        for (j++; j < k; j++) {
          w = __ldg(vw + j);
          if ((w >> 16) >= 2) break;
        }
        if (j < k) xa = wide::load_wf(tel(static_cast<int>(w >> 16) - 1, static_cast<int>(w & 0xffffu)));
        G = chain(G, xc);
      }
    } else {
      for (int j = 0; j < k; j++) {
        const uint32_t w = __ldg(vw + j);
        const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
        if (a >= 2) G = chain(G, wide::load_wf(tel(a - 1, v)));
      }
    }
    // Stage 2, forward: P_j = G x_{i_1} ... x_{i_j}; every kp.slot_stride-th
    // one is kept (slot j / stride), the others are recomputed below
    const int stride = kp.slot_stride;
    WV Pc = G;
    WF xf;
    if constexpr (Pf) xf = xw(vw, 0);
    for (int j = 0; j < k - 1; j++) {
      if (j % stride == 0) store_slot(slots, j / stride, lane, Pc);
      if constexpr (Pf) {
        const WF xc = xf;
        xf = xw(vw, j + 1);  // j + 1 <= k - 1
        Pc = chain(Pc, xc);
      } else {
        Pc = chain(Pc, xw(vw, j));
      }
    }
    const uint32_t wl = __ldg(vw + k - 1);
    const int vl = static_cast<int>(wl & 0xffffu), al = static_cast<int>(wl >> 16);
    WF xl;
    if constexpr (Pf)
      xl = xf;  // x_{i_k}
    else
      xl = wide::load_wf(tel(1, vl));
    f = add(f, wide::to_dd(wide::mul_x<false>(Pc, xl, c)));  // to_dd takes any leading bit
    accumulate_dd(jel(vl), c, valid, wide::to_dd(al == 1 ? Pc : wide::mul_small(Pc, static_cast<uint32_t>(al))));
    // Stage 2, backward.  With Pf the J entry of the next term is read one
    // term ahead: the positions of a monomial are distinct, so it is not the
    // entry this term writes.
    WV Q = wide::component(xl, c);
    norm = false;
    WF xb;
    double2 jb = make_double2(0.0, 0.0);
    if constexpr (Pf) {
      if (k >= 2) {
        const int v0 = static_cast<int>(__ldg(vw + k - 2) & 0xffffu);
        xb = wide::load_wf(tel(1, v0));
        jb = reinterpret_cast<const double2 *>(jel(v0))[c];
      }
    }
    for (int j = k - 2; j >= 0; j--) {
      const uint32_t w = __ldg(vw + j);
      const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
      WF xc;        // x_{i_j}
      double2 jc;   // J[p, i_j]
      if constexpr (Pf) {
        xc = xb;
        jc = jb;
        if (j > 0) {
          const int vn = static_cast<int>(__ldg(vw + j - 1) & 0xffffu);
          xb = wide::load_wf(tel(1, vn));
          jb = reinterpret_cast<const double2 *>(jel(vn))[c];
        }
      }
      WV Pj = load_slot(slots, j / stride, lane);
      for (int r = j - j % stride; r < j; r++) {  // recompute P_j from the kept P_{j - j % stride}
        if constexpr (Pf)
          Pj = wide::mul_x(Pj, r == j - 1 ? xb : xw(vw, r), c);
        else
          Pj = wide::mul_x(Pj, xw(vw, r), c);
      }
      const WV D = wide::mul_pair(Pj, Q, c);
      const dd term = wide::to_dd(a == 1 ? D : wide::mul_small(D, static_cast<uint32_t>(a)));
      if constexpr (Pf) {
        const dd sum = add(dd{jc.x, jc.y}, term);
        if (valid) reinterpret_cast<double2 *>(jel(v))[c] = make_double2(sum.h, sum.l);
        if (j > 0) Q = chain(Q, xc);
      } else {
        accumulate_dd(jel(v), c, valid, term);
        if (j > 0) Q = chain(Q, wide::load_wf(tel(1, v)));
      }
    }
  }
  if (valid) {
    const dd fo = normalize(f);
    reinterpret_cast<double2 *>(it.f_base + (static_cast<size_t>(sd.f_off) + static_cast<size_t>(pl) * Pz + q) * 4)[c] =
        make_double2(fo.h, fo.l);
    for (int v = 0; v < n; v++) {
      double2 *p = reinterpret_cast<double2 *>(jel(v)) + c;
      const double2 a = *p;
      const dd r = normalize(dd{a.x, a.y});
      *p = make_double2(r.h, r.l);
    }
  }
}

template <bool Pf>
__global__ void __launch_bounds__(kWarpsPerBlockMax * 32) main_wide(const MainParams kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *slots = reinterpret_cast<uint32_t *>(smem_raw) + static_cast<size_t>(warp) * kp.kslots * kSlotWords * 32;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(kp.counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (static_cast<int64_t>(item) >= kp.n_items) break;
    Item it;
    if (!decode_item(kp, item, lane, it)) continue;
    process_item_wide<Pf>(kp, it, slots, lane);
  }
}

cudaError_t convert_coef_wide(const double *coef_dd, uint32_t *coef_wide, int64_t M, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  int64_t blocks = (M + 255) / 256;
  if (blocks > kSms * 64) blocks = kSms * 64;
  convert_coef_kernel<<<static_cast<unsigned>(blocks), 256, 0, s>>>(coef_dd, coef_wide, M);
  return cudaGetLastError();
}

cudaError_t launch_powers_wide(const PowerParams &p, cudaStream_t s) {
  if (p.total <= 0) return cudaSuccess;
  int64_t blocks = (p.total + 127) / 128;
  if (blocks > kSms * 64) blocks = kSms * 64;
  powers_wide<<<static_cast<unsigned>(blocks), 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t prepare_main_wide(size_t smem_bytes) {
  const cudaError_t e =
      cudaFuncSetAttribute(main_wide<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_bytes));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(main_wide<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_bytes));
}

cudaError_t main_wide_occupancy(bool prefetch, int warps_per_block, size_t smem_bytes, int *blocks_per_sm) {
  return prefetch ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_wide<true>, warps_per_block * 32,
                                                                  smem_bytes)
                  : cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_wide<false>, warps_per_block * 32,
                                                                  smem_bytes);
}

cudaError_t launch_main_wide(const MainParams &p, int warps_per_block, size_t smem_bytes, int grid, cudaStream_t s) {
  if (p.n_items <= 0) return cudaSuccess;
  if (p.prefetch)
    main_wide<true><<<grid, warps_per_block * 32, smem_bytes, s>>>(p);
  else
    main_wide<false><<<grid, warps_per_block * 32, smem_bytes, s>>>(p);
  return cudaGetLastError();
}

}  // namespace pe
