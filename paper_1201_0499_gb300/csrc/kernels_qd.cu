// Kernels of the quad-double evaluation (precision PE_QD_INT): the method and
// work decomposition of kernels.cu (Sections 3.1-3.3 of the paper) with every
// product in the 256-bit block floating point of wide8.cuh and every sum in
// a 224-bit integer accumulator, so that the whole evaluation runs on the
// integer pipes.
//
//  * powers_qd: every point's variables converted to the block format and
//    their powers x^2 .. x^(d-1), in a table [e-1][n][P] of 80-byte entries
//    (entry e = 1 is x itself).
//  * main_qd: one warp per (polynomial, tile of 16 points, chunk of
//    monomials); lanes 2q and 2q+1 hold the real and the imaginary part of
//    point q.  Common factor with the coefficient folded in, forward products
//    in shared memory ([slot][word][lane]), value, backward running product,
//    derivatives; each term is added into the accumulator of its output
//    component: f in registers, the row J[p, :] in place in the output array
//    (an accumulator takes the 32 bytes of a quad-double component).
//  * finalize_qd: adds the accumulators of the chunks of a call and rounds
//    each sum to a quad-double, in place.
#include <cuda_runtime.h>

#include <cstdint>

#include "internal.h"
#include "items.cuh"
#include "wide8.cuh"

namespace pe {

using qd::Acc;
using qd::WF;
using qd::WV;

constexpr int kQdWords = kQdBytes / 4;  // 32-bit words per stored full value
constexpr int kQdSlotWords = 9;         // words per lane in a prefix-product slot (8 limbs, sign | exponent)
constexpr int kQdDoubles = 8;           // doubles per complex quad-double

__global__ void convert_coef_qd_kernel(const double *coef_qd, uint32_t *coef_blk, int64_t M) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < M; t += stride)
    qd::store_wf(coef_blk + t * kQdWords, qd::wf_from_cqd(coef_qd + t * kQdDoubles));
}

__global__ void powers_qd(const PowerParams pp) {
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
    const double *xp = pp.points + (pt_off + v * P + q) * kQdDoubles;
    auto entry = [&](int e) { return table + (tab_off + (static_cast<int64_t>(e - 1) * n + v) * P + q) * kQdWords; };
    const WF x = qd::wf_from_cqd(xp);
    qd::store_wf(entry(1), x);
    for (int e = 2; e < emax; e++) {
      const int h = e >> 1, g = e - h;
      const WF a = h == 1 ? x : qd::load_wf_coherent(entry(h));
      const WF b = g == 1 ? x : qd::load_wf_coherent(entry(g));
      qd::store_wf(entry(e), qd::wf_mul(b, a));
    }
  }
}

__device__ __forceinline__ void store_slot(uint32_t *slots, int j, int lane, const WV &v) {
  uint32_t *b = slots + j * (kQdSlotWords * 32) + lane;
#pragma unroll
  for (int i = 0; i < qd::L; i++) b[32 * i] = v.m.w[i];
  b[32 * qd::L] = v.s | (static_cast<uint32_t>(v.e) & 0x7fffffffu);  // exponents fit in 31 bits
}

__device__ __forceinline__ WV load_slot(const uint32_t *slots, int j, int lane) {
  const uint32_t *b = slots + j * (kQdSlotWords * 32) + lane;
  WV v;
#pragma unroll
  for (int i = 0; i < qd::L; i++) v.m.w[i] = b[32 * i];
  const uint32_t se = b[32 * qd::L];
  v.s = se & qd::kSignBit;
  v.e = static_cast<int32_t>(se << 1) >> 1;
  return v;
}

// Add a term into the accumulator of output component c of one entry.
__device__ __forceinline__ void accumulate(double *entry, int c, bool valid, const WV &t) {
  double *p = entry + 4 * c;
  Acc a = qd::load_acc(p);
  qd::acc_add(a, t);
  if (valid) qd::store_acc(p, a);
}

__device__ void process_item_qd(const MainParams &kp, const Item &it, uint32_t *slots, int lane) {
  const int gp = it.gp, tile = it.tile, s = it.s, P = it.P;
  const SysDesc sd = kp.sys[s];
  const int n = sd.n;
  const int q = tile * kPointsPerWarp + (lane >> 1);
  const bool valid = q < P;
  const int qc = valid ? q : P - 1;
  const int c = lane & 1;
  const size_t Pz = static_cast<size_t>(P);
  const int pl = gp - sd.poly0;
  const uint32_t *Tb = reinterpret_cast<const uint32_t *>(kp.table) + static_cast<size_t>(sd.tab_off) * kQdWords;
  const uint32_t *coef = reinterpret_cast<const uint32_t *>(kp.coef);
  double *Jrow = it.J_base + (static_cast<size_t>(sd.J_off) + static_cast<size_t>(pl) * n * Pz) * kQdDoubles;

  auto tel = [&](int e, int v) { return Tb + ((static_cast<size_t>(e - 1) * n + v) * Pz + qc) * kQdWords; };
  auto jel = [&](int v) { return Jrow + (static_cast<size_t>(v) * Pz + qc) * kQdDoubles; };

  if (valid)
    for (int v = 0; v < n; v++) qd::store_acc(jel(v) + 4 * c, qd::acc_zero());

  Acc f = qd::acc_zero();
  const int t0 = it.t0, t1 = it.t1;
  for (int t = t0; t < t1; t++) {
    const int vb = kp.mono_ptr[t];
    const int k = kp.mono_ptr[t + 1] - vb;
    WV G = qd::component(qd::load_wf(coef + static_cast<size_t>(t) * kQdWords), c);
    if (k == 0) {
      qd::acc_add(f, G);
      continue;
    }
    const uint32_t *vw = kp.var + vb;
    // Stage 1: G = c * prod_{a_j >= 2} x_{i_j}^(a_j - 1)
    for (int j = 0; j < k; j++) {
      const uint32_t w = __ldg(vw + j);
      const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
      if (a >= 2) G = qd::mul_x(G, qd::load_wf(tel(a - 1, v)), c);
    }
    // Stage 2, forward: P_j = G x_{i_1} ... x_{i_j}; every kp.slot_stride-th
    // one is kept (slot j / stride), the others are recomputed below
    const int stride = kp.slot_stride;
    WV Pc = G;
    for (int j = 0; j < k - 1; j++) {
      if (j % stride == 0) store_slot(slots, j / stride, lane, Pc);
      const int v = static_cast<int>(__ldg(vw + j) & 0xffffu);
      Pc = qd::mul_x(Pc, qd::load_wf(tel(1, v)), c);
    }
    const uint32_t wl = __ldg(vw + k - 1);
    const int vl = static_cast<int>(wl & 0xffffu), al = static_cast<int>(wl >> 16);
    const WF xl = qd::load_wf(tel(1, vl));
    qd::acc_add(f, qd::mul_x(Pc, xl, c));
    accumulate(jel(vl), c, valid, al == 1 ? Pc : qd::mul_small(Pc, static_cast<uint32_t>(al)));
    // Stage 2, backward
    WV Q = qd::component(xl, c);
    for (int j = k - 2; j >= 0; j--) {
      const uint32_t w = __ldg(vw + j);
      const int v = static_cast<int>(w & 0xffffu), a = static_cast<int>(w >> 16);
      WV Pj = load_slot(slots, j / stride, lane);
      for (int r = j - j % stride; r < j; r++)  // recompute P_j from the kept P_{j - j % stride}
        Pj = qd::mul_x(Pj, qd::load_wf(tel(1, static_cast<int>(__ldg(vw + r) & 0xffffu))), c);
      const WV D = qd::mul_pair(Pj, Q, c);
      accumulate(jel(v), c, valid, a == 1 ? D : qd::mul_small(D, static_cast<uint32_t>(a)));
      if (j > 0) Q = qd::mul_x(Q, qd::load_wf(tel(1, v)), c);
    }
  }
  if (valid) qd::store_acc(it.f_base + (static_cast<size_t>(sd.f_off) + static_cast<size_t>(pl) * Pz + q) * kQdDoubles + 4 * c, f);
}

__global__ void __launch_bounds__(kWarpsPerBlockMax * 32) main_qd(const MainParams kp) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *slots = reinterpret_cast<uint32_t *>(smem_raw) + static_cast<size_t>(warp) * kp.kslots * kQdSlotWords * 32;
  for (;;) {
    unsigned item = 0;
    if (lane == 0) item = atomicAdd(kp.counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (static_cast<int64_t>(item) >= kp.n_items) break;
    Item it;
    if (!decode_item(kp, item, lane, it)) continue;
    process_item_qd(kp, it, slots, lane);
  }
}

// One thread per output component (32 bytes): the sum of the chunks'
// accumulators, rounded to a quad-double in place.  `components` covers f
// (the first f_components) and then J.
__global__ void finalize_qd(double *out_f, double *out_J, const double *scratch_f, const double *scratch_J,
                            int64_t f_components, int64_t J_components, int chunks) {
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  const int64_t total = f_components + J_components;
  for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
    const bool isf = i < f_components;
    const int64_t j = isf ? i : i - f_components;
    double *p = (isf ? out_f : out_J) + j * 4;
    const double *sc = isf ? scratch_f : scratch_J;
    const int64_t cs = (isf ? f_components : J_components) * 4;  // doubles between chunk copies
    Acc a = qd::load_acc(p);
    for (int c = 1; c < chunks; c++) qd::acc_add_acc(a, qd::load_acc(sc + (c - 1) * cs + j * 4));
    double o[4];
    qd::acc_to_qd(a, o);
    reinterpret_cast<double2 *>(p)[0] = make_double2(o[0], o[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(o[2], o[3]);
  }
}

cudaError_t convert_coef_qd(const double *coef_qd, uint32_t *coef_blk, int64_t M, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  int64_t blocks = (M + 127) / 128;
  if (blocks > kSms * 32) blocks = kSms * 32;
  convert_coef_qd_kernel<<<static_cast<unsigned>(blocks), 128, 0, s>>>(coef_qd, coef_blk, M);
  return cudaGetLastError();
}

cudaError_t launch_powers_qd(const PowerParams &p, cudaStream_t s) {
  if (p.total <= 0) return cudaSuccess;
  int64_t blocks = (p.total + 127) / 128;
  if (blocks > kSms * 32) blocks = kSms * 32;
  powers_qd<<<static_cast<unsigned>(blocks), 128, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t prepare_main_qd(size_t smem_bytes) {
  return cudaFuncSetAttribute(main_qd, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_bytes));
}

cudaError_t main_qd_occupancy(int warps_per_block, size_t smem_bytes, int *blocks_per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, main_qd, warps_per_block * 32, smem_bytes);
}

cudaError_t launch_main_qd(const MainParams &p, int warps_per_block, size_t smem_bytes, int grid, cudaStream_t s) {
  if (p.n_items <= 0) return cudaSuccess;
  main_qd<<<grid, warps_per_block * 32, smem_bytes, s>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_finalize_qd(double *out_f, double *out_J, const double *scratch_f, const double *scratch_J,
                               int64_t f_components, int64_t J_components, int chunks, cudaStream_t s) {
  const int64_t total = f_components + J_components;
  if (total <= 0) return cudaSuccess;
  int64_t blocks = (total + 255) / 256;
  if (blocks > kSms * 16) blocks = kSms * 16;
  finalize_qd<<<static_cast<unsigned>(blocks), 256, 0, s>>>(out_f, out_J, scratch_f, scratch_J, f_components,
                                                            J_components, chunks);
  return cudaGetLastError();
}

}  // namespace pe
