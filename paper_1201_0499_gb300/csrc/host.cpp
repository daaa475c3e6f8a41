// Host side of the C ABI declared in include/polyeval.h: validation of a
// system in the format of Section 2 (Eq. 1), compilation into the device
// layout the kernels read, work lists, launches and handle lifetime.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "internal.h"
#include "polyeval.h"

using pe::SysDesc;

namespace {

constexpr int kMaxTimingEvents = 256;
// Splitting a polynomial's monomials into chunks (single-system calls with
// few (polynomial, tile) items): at most kMaxChunks chunks, partial results
// in at most kScratchBudget bytes of handle-owned scratch.
constexpr int kMaxChunks = 8;
constexpr size_t kScratchBudget = size_t{256} << 20;
// Integer double-double path: the largest slot stride tried (every
// stride-th forward product kept in shared memory, the others recomputed).
constexpr int kWideMaxStride = 3;
// Quad-double path: above this many prefix slots per lane a warp's 36-byte
// slots no longer leave room for 16 warps per SM, and only every second slot
// is stored.
constexpr int kQdSlotsFull = 12;

struct DeviceBuf {
  void *p = nullptr;
  size_t bytes = 0;
  ~DeviceBuf() {
    if (p) cudaFree(p);
  }
  int alloc(size_t b) {
    if (p) {
      cudaFree(p);
      p = nullptr;
      bytes = 0;
    }
    if (b == 0) return PE_OK;
    if (cudaMalloc(&p, b) != cudaSuccess) {
      cudaGetLastError();
      p = nullptr;
      return PE_ENOMEM;
    }
    bytes = b;
    return PE_OK;
  }
  template <class T>
  int upload(const std::vector<T> &v) {
    int rc = alloc(v.size() * sizeof(T));
    if (rc != PE_OK || v.empty()) return rc;
    return cudaMemcpy(p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess ? PE_OK : PE_ECUDA;
  }
};

}  // namespace

struct polyeval {
  bool dd = true;     // complex double-double points and outputs (PE_DD, PE_DD_INT)
  bool wide = false;  // products on the integer pipes (PE_DD_INT)
  bool qd = false;    // complex quad-double points and outputs, all on the integer pipes (PE_QD_INT)
  bool paper = false; // the paper's three-kernel design (PE_PAPER_KERNELS)
  int32_t paper_m = 0, paper_k = 0, paper_M = 0;
  bool batch = false;
  int32_t count = 0;
  int64_t max_points = 0;
  std::vector<SysDesc> sys;
  int32_t n_polys_total = 0;
  int32_t kmax = 0, kslots = 1;
  int32_t slot_stride = 1;  // integer path: keep every slot_stride-th forward product
  bool wide_prefetch = false;  // integer double-double path: the kernel that reads one step ahead
  int warps_per_block = pe::kWarpsPerBlockMax;
  size_t smem_bytes = 0;
  int blocks_per_sm = 1, sms = 1;
  int blocks_per_sm_1 = 1;  // occupancy with one warp per block
  size_t smem_per_warp = 0;
  int64_t n_items_batch = 0;
  int64_t f_total_batch = 0, J_total_batch = 0;  // batch: complex entries of all f and J
  int64_t power_total_batch = 0;
  double ops_per_point = 0.0, flops_per_point = 0.0;  // single: per point; batch: per whole evaluation
  // device memory
  DeviceBuf poly_ptr, mono_ptr, var, coef, coef_wide, poly_sys, sysd, perm, items, prefix, table, counter, status;
  DeviceBuf stage_pts, stage_f, stage_J;
  DeviceBuf scratch;  // chunk partial results (single-system handles)
  DeviceBuf paper_coeffs, paper_cf, paper_mons;  // three-kernel design
  // path tracking (single square systems): degrees of the polynomials and
  // the tracker's scratch, allocated on first use
  std::vector<int32_t> degrees;
  DeviceBuf deg_dev, tr_f, tr_J, tr_active, tr_x64, tr_status, tr_xc, tr_statc, tr_idx, tr_JL, tr_bL;
  // working copies of the paths (two, for compaction), their original
  // indices, the states of paths already written home, the running list
  DeviceBuf tr_xw[2], tr_xsw[2], tr_stw[2], tr_perm[2], tr_home, tr_list;
  DeviceBuf nt_Jdd, nt_fdd;  // quad-double Newton: double-double systems too large for shared memory
  cudaStream_t tr_stream = nullptr;  // the tracker's own stream (graph capture needs one)
  // polyeval_eval_host over point chunks: the copies of chunk c run on this
  // stream while chunk c + 1 is evaluated; two sets of staging buffers
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t chunk_done[2] = {}, chunk_copied[2] = {};
  struct Tuned {
    int64_t P;
    int chunks;
    int mode;    // 1: one single-warp block per item, 2: persistent grid
    int groups;  // monomial groups per warp (0: built-in choice)
  };
  std::vector<Tuned> tuned;  // launch choices found by polyeval_autotune, per point count
  // batch handles: the (polynomial, tile) work items in decreasing cost order
  // with the points of each tile, and the launch of polyeval_eval_many
  struct BatchTile {
    int32_t gp, tile, in_tile;
  };
  std::vector<BatchTile> btiles;
  int batch_gcap = pe::kPointsPerWarp;  // most monomial groups a partial tile may take
  int batch_chunks = 0, batch_mode = 0;  // 0: built-in choice
  // timing of the main kernel
  bool timing = false;
  cudaEvent_t ev[2 * kMaxTimingEvents] = {};
  int ev_used = 0, ev_dropped = 0;
  int64_t kernels_launched = 0;  // kernels queued by evals since timing was enabled
  ~polyeval() {
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
    if (tr_stream) cudaStreamDestroy(tr_stream);
    if (copy_stream) cudaStreamDestroy(copy_stream);
    for (auto &e : chunk_done)
      if (e) cudaEventDestroy(e);
    for (auto &e : chunk_copied)
      if (e) cudaEventDestroy(e);
  }
};

namespace {

int elem_doubles(const polyeval *h) { return h->qd ? 8 : h->dd ? 4 : 2; }

int ensure(DeviceBuf &b, size_t bytes) { return b.bytes >= bytes ? PE_OK : b.alloc(bytes); }

// Device arrays are read and written with 16-byte vector accesses.
bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool arrays_aligned(const void *a, const void *b, const void *c) {
  return aligned16(a) && aligned16(b) && aligned16(c);
}

// Products on the integer pipes (block-format table and coefficients).
bool block_format(const polyeval *h) { return h->wide || h->qd; }

// Table of powers: entries per (variable, point) and bytes per entry.  The
// double-double and double tables hold x^2 .. x^(emax-1); the block-format
// table also holds x itself (entry 1).
int64_t table_levels(const polyeval *h, int emax) {
  return block_format(h) ? std::max(emax - 1, 1) : std::max(emax - 2, 0);
}
size_t table_entry_bytes(const polyeval *h) {
  return h->qd ? pe::kQdBytes : h->wide ? pe::kWideBytes : elem_doubles(h) * sizeof(double);
}

// Launch the power-table kernel of the handle's precision.
int run_powers(polyeval *h, const pe::PowerParams &pp, cudaStream_t s) {
  const cudaError_t e = h->qd     ? pe::launch_powers_qd(pp, s)
                        : h->wide ? pe::launch_powers_wide(pp, s)
                                  : pe::launch_powers(h->dd, pp, s);
  if (e != cudaSuccess) return PE_ECUDA;
  if (pp.total > 0) h->kernels_launched++;
  return PE_OK;
}

// Bytes of one copy of f and J of a single-system call at P points.
size_t outputs_bytes(const polyeval *h, int64_t P) {
  const SysDesc &d = h->sys[0];
  return static_cast<size_t>(elem_doubles(h)) * sizeof(double) * static_cast<size_t>(P) *
         (static_cast<size_t>(d.N) + static_cast<size_t>(d.N) * d.n);
}

// Bytes of one copy of all f and J of a batch handle.
size_t batch_outputs_bytes(const polyeval *h) {
  return static_cast<size_t>(elem_doubles(h)) * sizeof(double) *
         static_cast<size_t>(h->f_total_batch + h->J_total_batch);
}

// The item table of a batch handle: (global polynomial, tile word) per item
// in decreasing cost order.  The tile word holds the tile index and log2 of
// the monomial groups of the item: a partial last tile with r < 16 points
// spreads them over the largest G <= gcap with G r <= 16 groups (double-double
// and double kernels; the integer-pipe kernels take one group).
std::vector<int32_t> batch_item_words(const polyeval *h, int gcap) {
  std::vector<int32_t> w;
  w.reserve(h->btiles.size() * 2);
  for (const polyeval::BatchTile &t : h->btiles) {
    int lg = 0;
    if (!block_format(h))
      while ((2 << lg) * t.in_tile <= pe::kPointsPerWarp && (2 << lg) <= gcap && lg < 4) lg++;
    w.push_back(t.gp);
    w.push_back(t.tile | (lg << pe::kTileBits));
  }
  return w;
}

// FP64 instructions and flops per point for one monomial (k variables, n2 of
// them with exponent >= 2), as the main kernel executes them (both lanes of
// a point).  Double-double, per lane: a chain product (common factor,
// forward and backward chains) is a dot product of 2 DMUL + 6 DFMA + 5 DADD
// = 13 instructions (19 flops), every kChainRenorm-th one renormalised by 3
// DADD more; a final product (value, derivatives) 13; a sum 5 DADD; an
// integer scale DMUL + 2 DFMA.  Double: a product DMUL + DFMA, a sum of J one
// DADD, a compensated sum of f 4 DADD, a scale one DMUL.
struct Cost {
  double ops = 0, flops = 0;
};

Cost monomial_cost(bool dd, int k, int n2) {
  if (k == 0) return dd ? Cost{10, 10} : Cost{8, 8};
  // chains: common factor + forward products (n2 + k - 1), backward (k - 2)
  const int l1 = n2 + k - 1, l2 = k >= 2 ? k - 2 : 0;
  const double renorm = l1 / pe::kChainRenorm + l2 / pe::kChainRenorm;
  const double plain = (l1 + l2) - renorm + (k >= 2 ? k : 1);  // + value and derivative products
  Cost c;
  if (dd) {
    c.ops = 32 * renorm + 26 * plain + 10 * (k + 1) + 6 * n2;
    c.flops = 44 * renorm + 38 * plain + 10 * (k + 1) + 10 * n2;
  } else {
    c.ops = 4 * (renorm + plain) + 2 * k + 8 + 2 * n2;
    c.flops = 6 * (renorm + plain) + 2 * k + 8 + 2 * n2;
  }
  return c;
}

// PE_DD_INT: only the double-double sums run on the FP64 pipe (5 DADD per
// lane per term); the products are integer instructions.
Cost monomial_cost_wide(int k) { return Cost{10.0 * (k + 1), 10.0 * (k + 1)}; }

// Per point and per polynomial: renormalising the row (double-double only)
// and finishing f.
Cost row_cost(bool dd, int n) { return dd ? Cost{6.0 * n + 6, 6.0 * n + 6} : Cost{2, 2}; }

// Per point and per variable: the powers x^2 .. x^(emax-1).
Cost power_cost(bool dd, int emax) {
  const double m = emax > 2 ? emax - 2 : 0;
  return dd ? Cost{32 * m, 44 * m} : Cost{4 * m, 6 * m};
}

// qd_coef: check the quad-double coefficients (coef_qd) instead of coef.
int validate(const pe_system *s, uint32_t flags, bool qd_coef) {
  if (!s || !s->poly_ptr || !s->mono_ptr) return PE_EINVAL;
  if (s->n_vars < 1 || s->n_polys < 0) return PE_EINVAL;
  if (s->n_vars > PE_MAX_VARS) return PE_ERANGE;
  if (s->poly_ptr[0] != 0) return PE_EINVAL;
  for (int32_t p = 0; p < s->n_polys; p++)
    if (s->poly_ptr[p + 1] < s->poly_ptr[p]) return PE_EINVAL;
  const int64_t M = s->poly_ptr[s->n_polys];
  if (M > INT32_MAX - 1) return PE_ERANGE;
  if (s->mono_ptr[0] != 0) return PE_EINVAL;
  for (int64_t t = 0; t < M; t++)
    if (s->mono_ptr[t + 1] < s->mono_ptr[t]) return PE_EINVAL;
  const int64_t nnz = s->mono_ptr[M];
  if (nnz > INT32_MAX - 1) return PE_ERANGE;
  if (nnz > 0 && (!s->pos || !s->exp)) return PE_EINVAL;
  if (M > 0 && !(qd_coef ? static_cast<const void *>(s->coef_qd) : static_cast<const void *>(s->coef)))
    return PE_EINVAL;
  for (int64_t t = 0; t < M; t++) {
    for (int64_t j = s->mono_ptr[t]; j < s->mono_ptr[t + 1]; j++) {
      if (s->pos[j] < 0 || s->pos[j] >= s->n_vars) return PE_EINVAL;
      if (j > s->mono_ptr[t] && s->pos[j] <= s->pos[j - 1]) return PE_EINVAL;
      if (s->exp[j] < 1) return PE_EINVAL;
      if (s->exp[j] > PE_MAX_EXP) return PE_ERANGE;
    }
    const double *c = qd_coef ? &s->coef_qd[t].re[0] : &s->coef[t].re_hi;
    const int nd = qd_coef ? 8 : 4;
    bool zero = true;
    for (int i = 0; i < nd; i++) {
      if (!std::isfinite(c[i])) return PE_EINVAL;
      zero = zero && c[i] == 0.0;
    }
    if (zero && !(flags & PE_ALLOW_ZERO_COEF)) return PE_EINVAL;
  }
  return PE_OK;
}

struct Compiled {
  std::vector<int32_t> poly_ptr{0}, mono_ptr{0}, poly_sys;
  std::vector<int32_t> poly_deg;  // total degree of each polynomial
  std::vector<uint32_t> var;
  std::vector<double> coef;
  std::vector<double> poly_ops, poly_flops;  // per point, per global polynomial
  int32_t kmax = 0;
};

int append_system(Compiled &c, const pe_system *s, int32_t sys_index, bool dd, bool wide, bool qd, SysDesc &d) {
  d.n = s->n_vars;
  d.N = s->n_polys;
  d.poly0 = static_cast<int32_t>(c.poly_sys.size());
  int32_t emax = 1;
  // PE_QD_INT executes no FP64 arithmetic; its polynomials are ordered by the
  // double-double cost, which grows with the same products and sums
  const Cost rc = row_cost(dd || qd, s->n_vars);
  for (int32_t p = 0; p < s->n_polys; p++) {
    Cost pc = rc;
    int32_t pdeg = 0;
    for (int64_t t = s->poly_ptr[p]; t < s->poly_ptr[p + 1]; t++) {
      const int64_t b = s->mono_ptr[t], e = s->mono_ptr[t + 1];
      int n2 = 0;
      int32_t mdeg = 0;
      for (int64_t j = b; j < e; j++) {
        const uint32_t a = static_cast<uint32_t>(s->exp[j]);
        c.var.push_back(static_cast<uint32_t>(s->pos[j]) | (a << 16));
        if (a >= 2) n2++;
        mdeg += static_cast<int32_t>(a);
        emax = std::max<int32_t>(emax, static_cast<int32_t>(a));
      }
      pdeg = std::max(pdeg, mdeg);
      const int k = static_cast<int>(e - b);
      c.kmax = std::max(c.kmax, k);
      const Cost mc = wide ? monomial_cost_wide(k) : monomial_cost(dd || qd, k, n2);
      pc.ops += mc.ops;
      pc.flops += mc.flops;
      if (c.var.size() > static_cast<size_t>(INT32_MAX - 1)) return PE_ERANGE;
      c.mono_ptr.push_back(static_cast<int32_t>(c.var.size()));
      if (qd) {
        // quad-double as given (the conversion kernel accepts any four
        // doubles per part), else the double-double widened with zeros
        if (s->coef_qd) {
          const pe_cqd &q = s->coef_qd[t];
          c.coef.insert(c.coef.end(), {q.re[0], q.re[1], q.re[2], q.re[3], q.im[0], q.im[1], q.im[2], q.im[3]});
        } else {
          const pe_cdd &q = s->coef[t];
          c.coef.insert(c.coef.end(), {q.re_hi, q.re_lo, 0.0, 0.0, q.im_hi, q.im_lo, 0.0, 0.0});
        }
        continue;
      }
      const pe_cdd &cf = s->coef[t];
      if (dd || wide) {
        // renormalised (FastTwoSum after ordering), so the first product of a
        // chain starts from |lo| <= ulp(hi)/2 whatever the caller passed
        auto renorm = [](double u, double w, double &hi, double &lo) {
          const double big = std::fabs(u) >= std::fabs(w) ? u : w, small = std::fabs(u) >= std::fabs(w) ? w : u;
          hi = big + small;
          lo = small - (hi - big);
        };
        double rh, rl, ih, il;
        renorm(cf.re_hi, cf.re_lo, rh, rl);
        renorm(cf.im_hi, cf.im_lo, ih, il);
        c.coef.insert(c.coef.end(), {rh, rl, ih, il});
      } else {
        c.coef.insert(c.coef.end(), {cf.re_hi, cf.im_hi});
      }
    }
    if (c.mono_ptr.size() > static_cast<size_t>(INT32_MAX - 1)) return PE_ERANGE;
    c.poly_ptr.push_back(static_cast<int32_t>(c.mono_ptr.size() - 1));
    c.poly_sys.push_back(sys_index);
    c.poly_deg.push_back(pdeg);
    c.poly_ops.push_back(pc.ops);
    c.poly_flops.push_back(pc.flops);
  }
  d.emax = emax;
  return PE_OK;
}

int finish_handle(polyeval *h, Compiled &c) {
  h->kmax = c.kmax;
  // forward products k - 1 per monomial; the grouped kernel also parks the k
  // derivative terms in the slots
  h->kslots = block_format(h) ? std::max(c.kmax - 1, 1) : std::max(c.kmax, 1);
  if (h->qd && h->kslots > kQdSlotsFull) {
    // keep every second forward product (the others are recomputed in the
    // backward pass) so that enough warps fit in shared memory
    h->slot_stride = 2;
    h->kslots = (h->kslots + 1) / 2;
  }
  h->n_polys_total = static_cast<int32_t>(c.poly_sys.size());
  int dev = 0, optin = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PE_ECUDA;
  if (cudaDeviceGetAttribute(&h->sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return PE_ECUDA;
  if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return PE_ECUDA;
  auto block_warps = [&](size_t pw) {
    int w = pe::kWarpsPerBlockMax;
    while (w > 1 && pw * w > static_cast<size_t>(optin)) w /= 2;
    return w;
  };
  if (h->wide) {
    // The integer kernel is bound by the latency of its carry chains, so
    // resident warps pay for recomputed products: take the slot stride
    // (1 .. kWideMaxStride) that leaves the most warps resident, the smallest
    // among equals.  Measured on GB300: n = 128, k = 32: stride 3 (32 warps
    // per SM) 4.43 K evaluations/s against 4.07 K with stride 2 (20 warps) and
    // 2.58 K with stride 1; n = 64, k = 16: stride 2 76.1 K, stride 1 71.5 K.
    if (pe::prepare_main_wide(static_cast<size_t>(optin)) != cudaSuccess) return PE_ECUDA;
    const int base = std::max(c.kmax - 1, 1);
    int best_w = -1;
    for (int st = 1; st <= kWideMaxStride; st++) {
      const int ks = (base + st - 1) / st;
      const size_t pw = static_cast<size_t>(ks) * 32 * pe::kWideSlotBytes;
      const int wpb = block_warps(pw);
      if (pw * wpb > static_cast<size_t>(optin)) continue;
      int blocks = 0;
      if (pe::main_wide_occupancy(false, wpb, pw * wpb, &blocks) != cudaSuccess) return PE_ECUDA;
      if (blocks * wpb > best_w) {
        best_w = blocks * wpb;
        h->slot_stride = st;
        h->kslots = ks;
      }
    }
    if (best_w < 0) return PE_ERANGE;
  }
  const size_t per_warp = static_cast<size_t>(h->kslots) * 32 *
                         (h->qd ? pe::kQdSlotBytes : h->wide ? pe::kWideSlotBytes : (h->dd ? 16 : 8));
  h->warps_per_block = block_warps(per_warp);
  if (per_warp * h->warps_per_block > static_cast<size_t>(optin)) return PE_ERANGE;
  h->smem_bytes = per_warp * h->warps_per_block;
  h->smem_per_warp = per_warp;
  if (h->qd) {
    if (pe::prepare_main_qd(static_cast<size_t>(optin)) != cudaSuccess) return PE_ECUDA;
    if (pe::main_qd_occupancy(h->warps_per_block, h->smem_bytes, &h->blocks_per_sm) != cudaSuccess) return PE_ECUDA;
    if (pe::main_qd_occupancy(1, per_warp, &h->blocks_per_sm_1) != cudaSuccess) return PE_ECUDA;
  } else if (h->wide) {
    // The kernel that reads one step ahead holds more registers: take it when
    // it keeps as many resident warps as the other (where shared memory, not
    // registers, limits residency; with the stride chosen above that is rare).
    int plain = 0, ahead = 0;
    if (pe::main_wide_occupancy(false, h->warps_per_block, h->smem_bytes, &plain) != cudaSuccess ||
        pe::main_wide_occupancy(true, h->warps_per_block, h->smem_bytes, &ahead) != cudaSuccess)
      return PE_ECUDA;
    h->wide_prefetch = ahead >= plain;
    h->blocks_per_sm = h->wide_prefetch ? ahead : plain;
    if (pe::main_wide_occupancy(h->wide_prefetch, 1, per_warp, &h->blocks_per_sm_1) != cudaSuccess) return PE_ECUDA;
  } else {
    if (pe::prepare_main(h->dd, static_cast<size_t>(optin)) != cudaSuccess) return PE_ECUDA;
    if (pe::main_occupancy(h->dd, h->batch, h->warps_per_block, h->smem_bytes, &h->blocks_per_sm) != cudaSuccess)
      return PE_ECUDA;
    if (pe::main_occupancy(h->dd, h->batch, 1, per_warp, &h->blocks_per_sm_1) != cudaSuccess) return PE_ECUDA;
  }
  if (h->blocks_per_sm < 1 || h->blocks_per_sm_1 < 1) return PE_ERANGE;
  int rc;
  if ((rc = h->poly_ptr.upload(c.poly_ptr)) || (rc = h->mono_ptr.upload(c.mono_ptr)) || (rc = h->var.upload(c.var)) ||
      (rc = h->coef.upload(c.coef)) || (rc = h->poly_sys.upload(c.poly_sys)) || (rc = h->sysd.upload(h->sys)))
    return rc;
  if ((rc = h->counter.alloc(sizeof(unsigned))) || (rc = h->status.alloc(sizeof(int)))) return rc;
  if (cudaMemset(h->status.p, 0, sizeof(int)) != cudaSuccess) return PE_ECUDA;
  if (block_format(h)) {  // coefficients to the block format, once
    const int64_t M = static_cast<int64_t>(c.coef.size() / (h->qd ? 8 : 4));
    if ((rc = h->coef_wide.alloc(static_cast<size_t>(M) * (h->qd ? pe::kQdBytes : pe::kWideBytes))) != PE_OK)
      return rc;
    const cudaError_t ce =
        h->qd ? pe::convert_coef_qd(static_cast<const double *>(h->coef.p), static_cast<uint32_t *>(h->coef_wide.p), M,
                                    nullptr)
              : pe::convert_coef_wide(static_cast<const double *>(h->coef.p), static_cast<uint32_t *>(h->coef_wide.p),
                                      M, nullptr);
    if (ce != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return PE_ECUDA;
    h->coef.alloc(0);
  }
  return PE_OK;
}

// Launch shape.  When every item fits in one wave of resident warps, launch
// one single-warp block per item: the block scheduler then spreads the warps
// over the SMs to within one warp, which balances the FP64 pipe of every SM.
// Otherwise a persistent grid of full blocks takes items from the counter.
struct Shape {
  int grid, warps;
  size_t smem;
};

Shape shape_for(const polyeval *h, int64_t n_items, int mode = 0) {
  if (mode == 1 || (mode == 0 && n_items <= static_cast<int64_t>(h->sms) * h->blocks_per_sm_1))
    return Shape{static_cast<int>(std::max<int64_t>(1, n_items)), 1, h->smem_per_warp};
  const int64_t full = static_cast<int64_t>(h->sms) * h->blocks_per_sm;
  const int64_t need = (n_items + h->warps_per_block - 1) / h->warps_per_block;
  return Shape{static_cast<int>(std::max<int64_t>(1, std::min(full, need))), h->warps_per_block, h->smem_bytes};
}

// x * k for a double-double x and a small integer k (TwoProd with an FMA on
// the high word), renormalised.
void dd_times_int(double hi, double lo, double k, double &rh, double &rl) {
  const double p = hi * k;
  const double e = std::fma(hi, k, -p);
  const double t = std::fma(lo, k, e);
  rh = p + t;
  rl = t - (rh - p);
}

// The paper's layout: Coeffs holds, for each variable position j of the
// monomials in S_m order, the coefficients c a_j of the derivatives, then the
// coefficients c themselves (Section 3.3).
int setup_paper(polyeval *h, const pe_system *sys, const Compiled &c) {
  if (!h->dd || h->wide || h->qd) return PE_EINVAL;
  const SysDesc &d = h->sys[0];
  if (d.N < 1 || h->max_points > 65535) return PE_EINVAL;
  const int64_t M = sys->poly_ptr[d.N];
  const int64_t m = sys->poly_ptr[1] - sys->poly_ptr[0];
  if (m < 1) return PE_EINVAL;
  for (int32_t p = 0; p < d.N; p++)
    if (sys->poly_ptr[p + 1] - sys->poly_ptr[p] != m) return PE_EINVAL;
  const int64_t k = sys->mono_ptr[1] - sys->mono_ptr[0];
  if (k < 3) return PE_EINVAL;
  for (int64_t t = 0; t < M; t++)
    if (sys->mono_ptr[t + 1] - sys->mono_ptr[t] != k) return PE_EINVAL;
  h->paper = true;
  h->paper_m = static_cast<int32_t>(m);
  h->paper_k = static_cast<int32_t>(k);
  h->paper_M = static_cast<int32_t>(M);
  std::vector<double> co(static_cast<size_t>(k + 1) * M * 4);
  for (int64_t t = 0; t < M; t++) {
    const double *cf = &c.coef[static_cast<size_t>(t) * 4];
    for (int64_t j = 0; j <= k; j++) {
      const double a = j < k ? static_cast<double>(sys->exp[sys->mono_ptr[t] + j]) : 1.0;
      double *dst = &co[(static_cast<size_t>(j) * M + t) * 4];
      dd_times_int(cf[0], cf[1], a, dst[0], dst[1]);
      dd_times_int(cf[2], cf[3], a, dst[2], dst[3]);
    }
  }
  int rc;
  const size_t slots = static_cast<size_t>(d.N) * (d.n + 1);
  if ((rc = h->paper_coeffs.upload(co)) != PE_OK) return rc;
  if ((rc = h->paper_cf.alloc(static_cast<size_t>(h->max_points) * M * 32)) != PE_OK) return rc;
  if ((rc = h->paper_mons.alloc(static_cast<size_t>(h->max_points) * m * slots * 32)) != PE_OK) return rc;
  if (cudaMemset(h->paper_mons.p, 0, h->paper_mons.bytes) != cudaSuccess) return PE_ECUDA;  // zero terms, once
  int optin = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
    return PE_ECUDA;
  const size_t sm1 = 32 * static_cast<size_t>(d.n) * std::max(d.emax - 1, 1);
  const size_t sm2 = 32 * (static_cast<size_t>(d.n) + static_cast<size_t>(k + 2) * 32);
  if (sm1 > static_cast<size_t>(optin) || sm2 > static_cast<size_t>(optin)) return PE_ERANGE;
  if (pe::prepare_paper(static_cast<size_t>(optin), static_cast<size_t>(optin)) != cudaSuccess) return PE_ECUDA;
  // work of the paper's method per point: K1 powers per block of 32 and k-1
  // products per monomial, K2 5k-4 products, K3 (n^2+n) m sums; a complex
  // double-double product is 32 FP64 instructions (44 flops), a sum 10
  const double blocks = static_cast<double>((M + 31) / 32);
  const double cm = blocks * d.n * std::max(d.emax - 2, 0) + static_cast<double>(M) * (k - 1) +
                    static_cast<double>(M) * (5 * k - 4);
  const double ca = static_cast<double>(slots) * m;
  h->ops_per_point = 32 * cm + 10 * ca;
  h->flops_per_point = 44 * cm + 10 * ca;
  return PE_OK;
}

pe::MainParams main_params(const polyeval *h) {
  pe::MainParams p{};
  p.poly_ptr = static_cast<const int32_t *>(h->poly_ptr.p);
  p.mono_ptr = static_cast<const int32_t *>(h->mono_ptr.p);
  p.var = static_cast<const uint32_t *>(h->var.p);
  p.coef = static_cast<const double *>(block_format(h) ? h->coef_wide.p : h->coef.p);
  p.poly_sys = static_cast<const int32_t *>(h->poly_sys.p);
  p.sys = static_cast<const SysDesc *>(h->sysd.p);
  p.perm = static_cast<const int32_t *>(h->perm.p);
  p.items = static_cast<const int2 *>(h->items.p);
  p.table = static_cast<const double *>(h->table.p);
  p.kslots = h->kslots;
  p.tile_points = pe::kPointsPerWarp;
  p.groups = 1;
  p.slot_stride = h->slot_stride;
  p.prefetch = h->wide_prefetch ? 1 : 0;
  p.n_polys_total = h->n_polys_total;
  p.counter = static_cast<unsigned *>(h->counter.p);
  p.status = static_cast<int *>(h->status.p);
  return p;
}

int run_main(polyeval *h, const pe::MainParams &mp, cudaStream_t s, int mode = 0) {
  if (mp.n_items <= 0) return PE_OK;
  if (cudaMemsetAsync(h->counter.p, 0, sizeof(unsigned), s) != cudaSuccess) return PE_ECUDA;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->timing) {
    if (h->ev_used < kMaxTimingEvents) {
      e0 = h->ev[2 * h->ev_used];
      e1 = h->ev[2 * h->ev_used + 1];
      h->ev_used++;
    } else {
      h->ev_dropped++;
    }
  }
  if (e0 && cudaEventRecord(e0, s) != cudaSuccess) return PE_ECUDA;
  const Shape sh = shape_for(h, mp.n_items, mode);
  const cudaError_t le = h->qd     ? pe::launch_main_qd(mp, sh.warps, sh.smem, sh.grid, s)
                         : h->wide ? pe::launch_main_wide(mp, sh.warps, sh.smem, sh.grid, s)
                                   : pe::launch_main(h->dd, mp, sh.warps, sh.smem, sh.grid, s);
  if (le != cudaSuccess) return PE_ECUDA;
  h->kernels_launched++;
  if (e1 && cudaEventRecord(e1, s) != cudaSuccess) return PE_ECUDA;
  return PE_OK;
}

}  // namespace

extern "C" {

int polyeval_validate(const pe_system *sys, uint32_t flags) {
  return validate(sys, flags, sys && !sys->coef && sys->coef_qd);
}

}  // extern "C"

namespace {

bool valid_precision(int precision) {
  return precision == PE_DD || precision == PE_F64 || precision == PE_DD_INT || precision == PE_QD_INT;
}

void set_precision(polyeval *h, int precision) {
  h->dd = precision != PE_F64;
  h->wide = precision == PE_DD_INT;
  h->qd = precision == PE_QD_INT;
}

}  // namespace

extern "C" {


int polyeval_create(const pe_system *sys, int precision, uint32_t flags, int64_t max_points, polyeval_t **out) {
  if (!out) return PE_EINVAL;
  *out = nullptr;
  if (!valid_precision(precision)) return PE_EINVAL;
  if (max_points < 1) return PE_EINVAL;
  int rc = validate(sys, flags, sys && precision == PE_QD_INT && sys->coef_qd);
  if (rc != PE_OK) return rc;
  polyeval *h = nullptr;
  try {
    h = new polyeval();
    set_precision(h, precision);
    h->batch = false;
    h->count = 1;
    h->max_points = max_points;
    h->sys.resize(1);
    Compiled c;
    if ((rc = append_system(c, sys, 0, h->dd, h->wide, h->qd, h->sys[0])) != PE_OK) {
      delete h;
      return rc;
    }
    SysDesc &d = h->sys[0];
    const int64_t tiles = (max_points + pe::kPointsPerWarp - 1) / pe::kPointsPerWarp;
    if (static_cast<int64_t>(d.N) * tiles > INT32_MAX || max_points > INT32_MAX) {
      delete h;
      return PE_ERANGE;
    }
    d.P = 0;
    d.tiles = 0;
    d.pt_off = d.f_off = d.J_off = d.tab_off = 0;
    // polynomials by decreasing cost (largest first), stable
    std::vector<int32_t> perm(d.N);
    std::iota(perm.begin(), perm.end(), 0);
    std::stable_sort(perm.begin(), perm.end(), [&](int32_t a, int32_t b) { return c.poly_ops[a] > c.poly_ops[b]; });
    double ops = 0, flops = 0;
    for (int32_t p = 0; p < d.N; p++) {
      ops += c.poly_ops[p];
      flops += c.poly_flops[p];
    }
    const Cost pw = block_format(h) ? Cost{} : power_cost(h->dd, d.emax);
    h->ops_per_point = h->qd ? 0.0 : ops + pw.ops * d.n;
    h->flops_per_point = h->qd ? 0.0 : flops + pw.flops * d.n;
    if ((rc = finish_handle(h, c)) != PE_OK || (rc = h->perm.upload(perm)) != PE_OK) {
      delete h;
      return rc;
    }
    h->degrees = c.poly_deg;
    if (flags & PE_PAPER_KERNELS) {
      if ((rc = setup_paper(h, sys, c)) != PE_OK) {
        delete h;
        return rc;
      }
    }
    {
      const size_t per_chunk = outputs_bytes(h, max_points);
      const size_t want = std::min(static_cast<size_t>(kMaxChunks - 1) * per_chunk, kScratchBudget);
      if (per_chunk > 0 && want >= per_chunk && (rc = h->scratch.alloc(want)) != PE_OK) {
        delete h;
        return rc;
      }
    }
    const int64_t levels = table_levels(h, d.emax);
    if (levels > 0) {
      const size_t entries = static_cast<size_t>(levels) * d.n * static_cast<size_t>(max_points);
      if ((rc = h->table.alloc(entries * table_entry_bytes(h))) != PE_OK) {
        delete h;
        return rc;
      }
    }
  } catch (const std::bad_alloc &) {
    delete h;
    return PE_ENOMEM;
  }
  *out = h;
  return PE_OK;
}

int polyeval_create_many(const pe_system *systems, int32_t count, int precision, uint32_t flags,
                         const int64_t *points_per_system, polyeval_t **out) {
  if (!out) return PE_EINVAL;
  *out = nullptr;
  if (!systems || !points_per_system || count < 1) return PE_EINVAL;
  if (!valid_precision(precision)) return PE_EINVAL;
  for (int32_t s = 0; s < count; s++) {
    int rc = validate(&systems[s], flags, precision == PE_QD_INT && systems[s].coef_qd);
    if (rc != PE_OK) return rc;
    if (points_per_system[s] < 0 || points_per_system[s] > INT32_MAX) return PE_EINVAL;
  }
  polyeval *h = nullptr;
  int rc = PE_OK;
  try {
    h = new polyeval();
    set_precision(h, precision);
    h->batch = true;
    h->count = count;
    h->sys.resize(count);
    Compiled c;
    int64_t pt = 0, fo = 0, jo = 0, to = 0;
    std::vector<int64_t> prefix{0};
    struct Item {
      int32_t gp, tile, in_tile;
      double cost;
    };
    std::vector<Item> items;
    double ops = 0, flops = 0;
    for (int32_t s = 0; s < count; s++) {
      SysDesc &d = h->sys[s];
      if ((rc = append_system(c, &systems[s], s, h->dd, h->wide, h->qd, d)) != PE_OK) {
        delete h;
        return rc;
      }
      const int64_t P = points_per_system[s];
      d.P = static_cast<int32_t>(P);
      d.tiles = static_cast<int32_t>((P + pe::kPointsPerWarp - 1) / pe::kPointsPerWarp);
      d.pt_off = pt;
      d.f_off = fo;
      d.J_off = jo;
      d.tab_off = to;
      pt += static_cast<int64_t>(d.n) * P;
      fo += static_cast<int64_t>(d.N) * P;
      jo += static_cast<int64_t>(d.N) * d.n * P;
      const bool tab = table_levels(h, d.emax) > 0 && P > 0;
      to += tab ? table_levels(h, d.emax) * d.n * P : 0;
      prefix.push_back(prefix.back() + (tab ? static_cast<int64_t>(d.n) * P : 0));
      const Cost pw = block_format(h) ? Cost{} : power_cost(h->dd, d.emax);
      ops += pw.ops * d.n * P;
      flops += pw.flops * d.n * P;
      for (int32_t p = 0; p < d.N; p++) {
        const int32_t gp = d.poly0 + p;
        ops += c.poly_ops[gp] * P;
        flops += c.poly_flops[gp] * P;
        for (int32_t tl = 0; tl < d.tiles; tl++) {
          const int32_t in_tile = static_cast<int32_t>(std::min<int64_t>(pe::kPointsPerWarp, P - tl * pe::kPointsPerWarp));
          items.push_back(Item{gp, tl, in_tile, c.poly_ops[gp] * in_tile});
        }
      }
    }
    if (items.size() > static_cast<size_t>(INT32_MAX)) {
      delete h;
      return PE_ERANGE;
    }
    std::stable_sort(items.begin(), items.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
    h->btiles.reserve(items.size());
    for (const Item &it : items) h->btiles.push_back(polyeval::BatchTile{it.gp, it.tile, it.in_tile});
    const std::vector<int32_t> it2 = batch_item_words(h, h->batch_gcap);
    h->n_items_batch = static_cast<int64_t>(items.size());
    h->power_total_batch = prefix.back();
    h->f_total_batch = fo;
    h->J_total_batch = jo;
    h->ops_per_point = h->qd ? 0.0 : ops;
    h->flops_per_point = h->qd ? 0.0 : flops;
    if ((rc = finish_handle(h, c)) != PE_OK || (rc = h->items.upload(it2)) != PE_OK ||
        (rc = h->prefix.upload(prefix)) != PE_OK ||
        (rc = h->table.alloc(static_cast<size_t>(to) * table_entry_bytes(h))) != PE_OK) {
      delete h;
      return rc;
    }
    {  // scratch for monomial chunks of batches with few work items
      const size_t per_chunk = batch_outputs_bytes(h);
      const size_t want = std::min(static_cast<size_t>(kMaxChunks - 1) * per_chunk, kScratchBudget);
      if (per_chunk > 0 && want >= per_chunk && (rc = h->scratch.alloc(want)) != PE_OK) {
        delete h;
        return rc;
      }
    }
  } catch (const std::bad_alloc &) {
    delete h;
    return PE_ENOMEM;
  }
  *out = h;
  return PE_OK;
}

int polyeval_many_layout(const polyeval_t *h, int32_t s, int64_t *pt_off, int64_t *f_off, int64_t *J_off) {
  if (!h || !h->batch || s < 0 || s > h->count) return PE_EINVAL;
  int64_t a, b, c;
  if (s < h->count) {
    a = h->sys[s].pt_off;
    b = h->sys[s].f_off;
    c = h->sys[s].J_off;
  } else {
    const SysDesc &d = h->sys[h->count - 1];
    a = d.pt_off + static_cast<int64_t>(d.n) * d.P;
    b = d.f_off + static_cast<int64_t>(d.N) * d.P;
    c = d.J_off + static_cast<int64_t>(d.N) * d.n * d.P;
  }
  if (pt_off) *pt_off = a;
  if (f_off) *f_off = b;
  if (J_off) *J_off = c;
  return PE_OK;
}

}  // extern "C"

namespace {

// One single-system evaluation.  chunks > 0 and mode > 0 force the monomial
// chunk count and the launch shape (used by the autotuner); 0 picks them from
// the tuned table or the heuristic.
// Monomial groups per warp for P points: enough that the lane pairs of a warp
// are busy when P < 16 (the largest power of two G with G P <= 16).
// Point chunks of polyeval_eval_host: one per 256 MiB of outputs, at most 8,
// each of at least 1024 points (a chunk's evaluation then still fills the GPU).
int host_chunks(const polyeval *h, int64_t P) {
  const SysDesc &d = h->sys[0];
  const size_t out = static_cast<size_t>(elem_doubles(h)) * sizeof(double) * static_cast<size_t>(P) *
                     (static_cast<size_t>(d.N) + static_cast<size_t>(d.N) * d.n);
  int C = static_cast<int>(std::min<size_t>(8, out >> 28));
  while (C > 1 && P / C < 1024) C--;
  return std::max(C, 1);
}

int default_groups(int64_t P) {
  int G = 1;
  while (G < 16 && 2 * G * P <= pe::kPointsPerWarp) G *= 2;
  return G;
}

int eval_single(polyeval *h, const void *points, int64_t P, void *out_f, void *out_J, cudaStream_t s, int chunks,
                int mode, int groups = 0) {
  if (!h || h->batch || P < 0) return PE_EINVAL;
  if (P == 0) return PE_OK;
  if (P > h->max_points) return PE_ERANGE;
  if (!points || (!out_f && h->sys[0].N > 0) || (!out_J && h->sys[0].N > 0)) return PE_EINVAL;
  if (!arrays_aligned(points, out_f, out_J)) return PE_EINVAL;
  const SysDesc &d = h->sys[0];
  if (h->paper) {
    pe::PaperParams pp{};
    pp.n = d.n;
    pp.N = d.N;
    pp.M = h->paper_M;
    pp.m = h->paper_m;
    pp.k = h->paper_k;
    pp.d = d.emax;
    pp.P = static_cast<int32_t>(P);
    pp.var = static_cast<const uint32_t *>(h->var.p);
    pp.coeffs = static_cast<const double *>(h->paper_coeffs.p);
    pp.cf = static_cast<double *>(h->paper_cf.p);
    pp.mons = static_cast<double *>(h->paper_mons.p);
    pp.points = static_cast<const double *>(points);
    pp.out_f = static_cast<double *>(out_f);
    pp.out_J = static_cast<double *>(out_J);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->timing && h->ev_used < kMaxTimingEvents) {
      e0 = h->ev[2 * h->ev_used];
      e1 = h->ev[2 * h->ev_used + 1];
      h->ev_used++;
    }
    if (e0 && cudaEventRecord(e0, s) != cudaSuccess) return PE_ECUDA;
    if (pe::launch_paper(pp, s) != cudaSuccess) return PE_ECUDA;
    if (e1 && cudaEventRecord(e1, s) != cudaSuccess) return PE_ECUDA;
    h->kernels_launched += 3;
    return PE_OK;
  }
  if (table_levels(h, d.emax) > 0) {
    pe::PowerParams pp{};
    pp.sys = static_cast<const SysDesc *>(h->sysd.p);
    pp.points = static_cast<const double *>(points);
    pp.table = static_cast<double *>(h->table.p);
    pp.total = static_cast<int64_t>(d.n) * P;
    pp.count = 1;
    pp.single_P = static_cast<int32_t>(P);
    pp.single_n = d.n;
    pp.single_emax = d.emax;
    if (run_powers(h, pp, s) != PE_OK) return PE_ECUDA;
  }
  pe::MainParams mp = main_params(h);
  mp.points = static_cast<const double *>(points);
  mp.out_f = static_cast<double *>(out_f);
  mp.out_J = static_cast<double *>(out_J);
  mp.single_P = static_cast<int32_t>(P);
  if (chunks <= 0 || mode <= 0 || groups <= 0) {
    for (const auto &t : h->tuned)
      if (t.P == P) {
        if (chunks <= 0) chunks = t.chunks;
        if (mode <= 0) mode = t.mode;
        if (groups <= 0) groups = t.groups;
      }
  }
  // monomial groups per warp (double-double and double kernels only)
  int G = block_format(h) ? 1 : (groups > 0 ? groups : default_groups(P));
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16) G = 1;
  mp.groups = G;
  mp.tile_points = pe::kPointsPerWarp / G;
  mp.single_T = static_cast<int32_t>((P + mp.tile_points - 1) / mp.tile_points);
  const int64_t base = static_cast<int64_t>(d.N) * mp.single_T;
  // Few (polynomial, tile) items: split each polynomial's monomials into
  // chunks so that about one wave of resident warps has work.
  int C = 1;
  const int64_t capacity = static_cast<int64_t>(h->sms) * h->blocks_per_sm_1;
  const size_t per_chunk = outputs_bytes(h, P);
  if (base > 0 && per_chunk > 0) {
    // about one wave of items; the quad-double kernel, whose long carry
    // chains leave it latency bound, gains from about two (measured: 4
    // chunks 1.98 ms, 1 chunk 2.38 ms on n = 32, m = 64, k = 9, 1024 points)
    const int64_t target = h->qd ? 2 * capacity : capacity;
    C = chunks > 0 ? std::min(chunks, kMaxChunks)
                   : static_cast<int>(std::min<int64_t>(kMaxChunks, std::max<int64_t>(1, target / base)));
    C = static_cast<int>(std::min<int64_t>(C, 1 + static_cast<int64_t>(h->scratch.bytes / per_chunk)));
  }
  const int64_t f_doubles = static_cast<int64_t>(elem_doubles(h)) * d.N * P;
  const int64_t J_doubles = f_doubles * d.n;
  mp.n_chunks = C;
  mp.chunk_f_stride = f_doubles;
  mp.chunk_J_stride = J_doubles;
  mp.scratch_f = static_cast<double *>(h->scratch.p);
  mp.scratch_J = C > 1 ? mp.scratch_f + static_cast<size_t>(C - 1) * f_doubles : nullptr;
  mp.n_items = base * C;
  if (mp.n_items > INT32_MAX) return PE_ERANGE;  // the work counter is 32-bit
  int rc = run_main(h, mp, s, mode);
  if (rc != PE_OK) return rc;
  if (h->qd) {  // add the chunks' accumulators, round to quad-double
    if (base > 0 && pe::launch_finalize_qd(mp.out_f, mp.out_J, mp.scratch_f, mp.scratch_J, 2 * static_cast<int64_t>(d.N) * P,
                                           2 * static_cast<int64_t>(d.N) * d.n * P, C, s) != cudaSuccess)
      return PE_ECUDA;
    if (base > 0) h->kernels_launched++;
    return PE_OK;
  }
  if (C == 1) return rc;
  if (pe::launch_combine(h->dd, mp.out_f, mp.out_J, mp.scratch_f, mp.scratch_J, f_doubles, J_doubles, C, s) !=
      cudaSuccess)
    return PE_ECUDA;
  h->kernels_launched += 2;  // f and J passes
  return PE_OK;
}

// One batch evaluation.  chunks > 0 and mode > 0 force the monomial chunk
// count and the launch shape (the autotuner); 0 takes the handle's choice,
// else the built-in one (one chunk; the shape from the item count).
int eval_many(polyeval *h, const void *points, void *out_f, void *out_J, cudaStream_t s, int chunks, int mode) {
  if (!h || !h->batch) return PE_EINVAL;
  if (h->n_items_batch == 0) return PE_OK;
  if (!points || !out_f || !out_J || !arrays_aligned(points, out_f, out_J)) return PE_EINVAL;
  if (h->power_total_batch > 0) {
    pe::PowerParams pp{};
    pp.sys = static_cast<const SysDesc *>(h->sysd.p);
    pp.prefix = static_cast<const int64_t *>(h->prefix.p);
    pp.points = static_cast<const double *>(points);
    pp.table = static_cast<double *>(h->table.p);
    pp.total = h->power_total_batch;
    pp.count = h->count;
    pp.single_P = -1;
    if (run_powers(h, pp, s) != PE_OK) return PE_ECUDA;
  }
  if (chunks <= 0) chunks = h->batch_chunks;
  if (mode <= 0) mode = h->batch_mode;
  const size_t per_chunk = batch_outputs_bytes(h);
  int C = std::max(1, std::min(chunks, kMaxChunks));
  C = static_cast<int>(std::min<int64_t>(C, 1 + static_cast<int64_t>(per_chunk ? h->scratch.bytes / per_chunk : 0)));
  if (h->n_items_batch * C > INT32_MAX) C = 1;  // the work counter is 32-bit
  const int64_t f_doubles = static_cast<int64_t>(elem_doubles(h)) * h->f_total_batch;
  const int64_t J_doubles = static_cast<int64_t>(elem_doubles(h)) * h->J_total_batch;
  pe::MainParams mp = main_params(h);
  mp.points = static_cast<const double *>(points);
  mp.out_f = static_cast<double *>(out_f);
  mp.out_J = static_cast<double *>(out_J);
  mp.single_P = -1;
  mp.single_T = 0;
  mp.n_chunks = C;
  mp.chunk_f_stride = f_doubles;
  mp.chunk_J_stride = J_doubles;
  mp.scratch_f = static_cast<double *>(h->scratch.p);
  mp.scratch_J = C > 1 ? mp.scratch_f + static_cast<size_t>(C - 1) * f_doubles : nullptr;
  mp.n_items = h->n_items_batch * C;
  const int rc = run_main(h, mp, s, std::max(mode, 0));
  if (rc != PE_OK) return rc;
  if (h->qd) {  // add the chunks' accumulators, round to quad-double
    if (pe::launch_finalize_qd(mp.out_f, mp.out_J, mp.scratch_f, mp.scratch_J, 2 * h->f_total_batch,
                               2 * h->J_total_batch, C, s) != cudaSuccess)
      return PE_ECUDA;
    h->kernels_launched++;
    return PE_OK;
  }
  if (C == 1) return PE_OK;
  if (pe::launch_combine(h->dd, mp.out_f, mp.out_J, mp.scratch_f, mp.scratch_J, f_doubles, J_doubles, C, s) !=
      cudaSuccess)
    return PE_ECUDA;
  h->kernels_launched += 2;  // f and J passes
  return PE_OK;
}

// Rewrites the batch item table for a cap on the monomial groups of partial
// tiles (after the work queued on every stream has finished).
int set_batch_gcap(polyeval *h, int gcap) {
  if (gcap == h->batch_gcap) return PE_OK;
  const std::vector<int32_t> w = batch_item_words(h, gcap);
  if (cudaDeviceSynchronize() != cudaSuccess) return PE_ECUDA;
  if (!w.empty() && cudaMemcpy(h->items.p, w.data(), w.size() * sizeof(int32_t), cudaMemcpyHostToDevice) != cudaSuccess)
    return PE_ECUDA;
  h->batch_gcap = gcap;
  return PE_OK;
}

// polyeval_autotune for a batch handle: monomial chunks (as the scratch
// allows), launch shape, and the cap on monomial groups of partial tiles
// (1: none; 16: as many as fill the warp).
int autotune_many(polyeval *h, const void *points, void *out_f, void *out_J, cudaStream_t s, int *chunks, int *shape,
                  int *groups) {
  if (!points || !out_f || !out_J || !arrays_aligned(points, out_f, out_J)) return PE_EINVAL;
  if (h->n_items_batch == 0) {  // nothing to time: report the launch in place
    if (chunks) *chunks = std::max(h->batch_chunks, 1);
    if (shape) *shape = h->batch_mode > 0 ? h->batch_mode : 2;
    if (groups) *groups = h->batch_gcap;
    return PE_OK;
  }
  const int64_t capacity = static_cast<int64_t>(h->sms) * h->blocks_per_sm_1;
  const size_t per_chunk = batch_outputs_bytes(h);
  const int max_c = per_chunk ? static_cast<int>(std::min<int64_t>(
                                    kMaxChunks, 1 + static_cast<int64_t>(h->scratch.bytes / per_chunk)))
                              : 1;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return PE_ECUDA;
  }
  const bool timing = h->timing;
  h->timing = false;
  float best = 0.0f;
  int best_c = 1, best_m = 2, best_g = h->batch_gcap;
  int rc = PE_OK;
  // the integer-pipe kernels take one group per item whatever the cap
  const int caps[2] = {block_format(h) ? 1 : pe::kPointsPerWarp, 1};
  for (int gi = 0; gi < (block_format(h) ? 1 : 2) && rc == PE_OK; gi++) {
    rc = set_batch_gcap(h, caps[gi]);
    for (int C = 1; C <= max_c && rc == PE_OK; C *= 2) {
      if (h->n_items_batch * C > INT32_MAX) continue;
      for (int m = 1; m <= 2 && rc == PE_OK; m++) {
        if (m == 1 && h->n_items_batch * C > capacity) continue;  // one wave only when every item is resident
        rc = eval_many(h, points, out_f, out_J, s, C, m);  // warm-up
        if (rc != PE_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = PE_ECUDA;
        for (int r = 0; r < 3 && rc == PE_OK; r++) rc = eval_many(h, points, out_f, out_J, s, C, m);
        if (rc == PE_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
          rc = PE_ECUDA;
        float ms = 0.0f;
        if (rc == PE_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PE_ECUDA;
        if (rc == PE_OK && (best == 0.0f || ms < best)) {
          best = ms;
          best_c = C;
          best_m = m;
          best_g = caps[gi];
        }
      }
    }
  }
  h->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PE_OK) return rc;
  if ((rc = set_batch_gcap(h, best_g)) != PE_OK) return rc;
  h->batch_chunks = best_c;
  h->batch_mode = best_m;
  // leave a valid evaluation with the chosen launch in the outputs
  if ((rc = eval_many(h, points, out_f, out_J, s, 0, 0)) != PE_OK) return rc;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PE_ECUDA;
  if (chunks) *chunks = best_c;
  if (shape) *shape = best_m;
  if (groups) *groups = best_g;
  return PE_OK;
}

}  // namespace

extern "C" {

int polyeval_eval(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream) {
  if (!h || h->batch || P < 0) return PE_EINVAL;
  if (P == 0) return PE_OK;
  if (P > h->max_points) return PE_ERANGE;
  if (!points || (!out_f && h->sys[0].N > 0) || (!out_J && h->sys[0].N > 0)) return PE_EINVAL;
  return eval_single(h, points, P, out_f, out_J, static_cast<cudaStream_t>(stream), 0, 0);
}

int polyeval_autotune(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream,
                      int *chunks, int *shape, int *groups) {
  if (h && h->batch) {
    if (P != 0) return PE_EINVAL;
    return autotune_many(h, points, out_f, out_J, static_cast<cudaStream_t>(stream), chunks, shape, groups);
  }
  if (!h || P < 1) return PE_EINVAL;
  if (P > h->max_points) return PE_ERANGE;
  if (!points || !out_f || !out_J || !arrays_aligned(points, out_f, out_J)) return PE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const SysDesc &d = h->sys[0];
  const int64_t capacity = static_cast<int64_t>(h->sms) * h->blocks_per_sm_1;
  const size_t per_chunk = outputs_bytes(h, P);
  const int max_c = per_chunk ? static_cast<int>(std::min<int64_t>(
                                    kMaxChunks, 1 + static_cast<int64_t>(h->scratch.bytes / per_chunk)))
                              : 1;
  // monomial groups: tried when the call has fewer points than 4 tiles
  const int max_g = block_format(h) || P >= 4 * pe::kPointsPerWarp ? 1 : 16;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return PE_ECUDA;
  }
  const bool timing = h->timing;
  h->timing = false;
  float best = 0.0f;
  int best_c = 1, best_m = 2, best_g = 1;
  int rc = PE_OK;
  for (int G = 1; G <= max_g && rc == PE_OK; G *= 2) {
    const int64_t tp = pe::kPointsPerWarp / G;
    const int64_t base = static_cast<int64_t>(d.N) * ((P + tp - 1) / tp);
    for (int C = 1; C <= max_c && rc == PE_OK; C *= 2) {
      if (base * C > INT32_MAX) continue;
      for (int m = 1; m <= 2 && rc == PE_OK; m++) {
        if (m == 1 && base * C > capacity) continue;  // one wave only when every item is resident
        rc = eval_single(h, points, P, out_f, out_J, s, C, m, G);  // warm-up
        if (rc != PE_OK) break;
        if (cudaEventRecord(e0, s) != cudaSuccess) rc = PE_ECUDA;
        for (int r = 0; r < 3 && rc == PE_OK; r++) rc = eval_single(h, points, P, out_f, out_J, s, C, m, G);
        if (rc == PE_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
          rc = PE_ECUDA;
        float ms = 0.0f;
        if (rc == PE_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = PE_ECUDA;
        if (rc == PE_OK && (best == 0.0f || ms < best)) {
          best = ms;
          best_c = C;
          best_m = m;
          best_g = G;
        }
      }
    }
  }
  h->timing = timing;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc != PE_OK) return rc;
  bool found = false;
  for (auto &t : h->tuned)
    if (t.P == P) {
      t.chunks = best_c;
      t.mode = best_m;
      t.groups = best_g;
      found = true;
    }
  if (!found) h->tuned.push_back(polyeval::Tuned{P, best_c, best_m, best_g});
  if (chunks) *chunks = best_c;
  if (shape) *shape = best_m;
  if (groups) *groups = best_g;
  return PE_OK;
}


int polyeval_set_launch(polyeval_t *h, int64_t P, int chunks, int shape, int groups) {
  if (!h || chunks < 0 || chunks > kMaxChunks || shape < 0 || shape > 2) return PE_EINVAL;
  if (groups != 0 && groups != 1 && groups != 2 && groups != 4 && groups != 8 && groups != 16) return PE_EINVAL;
  if (h->batch) {
    if (P != 0) return PE_EINVAL;
    const int rc = set_batch_gcap(h, groups > 0 ? groups : pe::kPointsPerWarp);
    if (rc != PE_OK) return rc;
    h->batch_chunks = chunks;
    h->batch_mode = shape;
    return PE_OK;
  }
  if (P < 1) return PE_EINVAL;
  for (auto it = h->tuned.begin(); it != h->tuned.end(); ++it)
    if (it->P == P) {
      h->tuned.erase(it);
      break;
    }
  if (chunks > 0 || shape > 0 || groups > 0) h->tuned.push_back(polyeval::Tuned{P, chunks, shape, groups});
  return PE_OK;
}

int polyeval_newton(polyeval_t *h, void *points, int64_t P, void *out_f, void *out_J, double *norms, void *stream) {
  if (!h || h->batch) return PE_EINVAL;
  const SysDesc &d = h->sys[0];
  if (d.N != d.n) return PE_EINVAL;
  if (h->qd && P > 0 && pe::newton_qd_needs_scratch(d.n)) {  // double-double systems of the solve
    const size_t np = static_cast<size_t>(d.n) * static_cast<size_t>(h->max_points);
    int r;
    if ((r = ensure(h->nt_Jdd, 32 * np * d.n)) || (r = ensure(h->nt_fdd, 32 * np))) return r;
  }
  int rc = polyeval_eval(h, points, P, out_f, out_J, stream);
  if (rc != PE_OK || P == 0) return rc;
  pe::NewtonParams np{};
  np.n = d.n;
  np.P = P;
  np.J = static_cast<double *>(out_J);
  np.f = static_cast<double *>(out_f);
  np.x = static_cast<double *>(points);
  np.norms = norms;
  np.Jdd = static_cast<double *>(h->nt_Jdd.p);
  np.fdd = static_cast<double *>(h->nt_fdd.p);
  const cudaError_t le = h->qd ? pe::launch_newton_qd(np, static_cast<cudaStream_t>(stream))
                               : pe::launch_newton(h->dd, np, static_cast<cudaStream_t>(stream));
  if (le != cudaSuccess) return PE_ECUDA;
  h->kernels_launched++;
  return PE_OK;
}

int polyeval_eval_many(polyeval_t *h, const void *points, void *out_f, void *out_J, void *stream) {
  return eval_many(h, points, out_f, out_J, static_cast<cudaStream_t>(stream), 0, 0);
}

int polyeval_eval_host(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream) {
  if (!h || h->batch || P < 0) return PE_EINVAL;
  if (P == 0) return PE_OK;
  if (P > h->max_points) return PE_ERANGE;
  if (!points || !out_f || !out_J) return PE_EINVAL;
  const SysDesc &d = h->sys[0];
  const size_t eb = static_cast<size_t>(elem_doubles(h)) * sizeof(double);
  const int C = host_chunks(h, P);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc;
  if (C == 1) {
    const size_t bp = eb * d.n * static_cast<size_t>(P), bf = eb * d.N * static_cast<size_t>(P),
                 bj = eb * d.N * static_cast<size_t>(d.n) * static_cast<size_t>(P);
    if ((rc = ensure(h->stage_pts, bp)) || (rc = ensure(h->stage_f, bf)) || (rc = ensure(h->stage_J, bj))) return rc;
    if (cudaMemcpyAsync(h->stage_pts.p, points, bp, cudaMemcpyHostToDevice, s) != cudaSuccess) return PE_ECUDA;
    if ((rc = polyeval_eval(h, h->stage_pts.p, P, h->stage_f.p, h->stage_J.p, stream)) != PE_OK) return rc;
    if (bf && cudaMemcpyAsync(out_f, h->stage_f.p, bf, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PE_ECUDA;
    if (bj && cudaMemcpyAsync(out_J, h->stage_J.p, bj, cudaMemcpyDeviceToHost, s) != cudaSuccess) return PE_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? PE_OK : PE_ECUDA;
  }
  // C chunks of at most Pc points, two staging sets used in turn: chunk c is
  // evaluated on `stream` while the outputs of chunk c - 1 go to the host on
  // the copy stream.  Each chunk's columns of the [.][P] host arrays are one
  // pitched copy.
  const int64_t Pc = (P + C - 1) / C;
  const size_t sp = eb * d.n * static_cast<size_t>(Pc), sf = eb * d.N * static_cast<size_t>(Pc),
               sj = eb * d.N * static_cast<size_t>(d.n) * static_cast<size_t>(Pc);
  if ((rc = ensure(h->stage_pts, 2 * sp)) || (rc = ensure(h->stage_f, 2 * sf)) || (rc = ensure(h->stage_J, 2 * sj)))
    return rc;
  if (!h->copy_stream && cudaStreamCreateWithFlags(&h->copy_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->copy_stream = nullptr;
    return PE_ECUDA;
  }
  for (int b = 0; b < 2; b++) {
    if (!h->chunk_done[b] && cudaEventCreateWithFlags(&h->chunk_done[b], cudaEventDisableTiming) != cudaSuccess)
      return PE_ECUDA;
    if (!h->chunk_copied[b] && cudaEventCreateWithFlags(&h->chunk_copied[b], cudaEventDisableTiming) != cudaSuccess)
      return PE_ECUDA;
  }
  const size_t hp = eb * static_cast<size_t>(P);  // row pitch of the host arrays
  rc = PE_OK;
  for (int c = 0; c < C && rc == PE_OK; c++) {
    const int64_t q0 = c * Pc, pc = std::min<int64_t>(Pc, P - q0);
    if (pc <= 0) break;
    const int b = c & 1;
    char *spts = static_cast<char *>(h->stage_pts.p) + b * sp;
    char *sff = static_cast<char *>(h->stage_f.p) + b * sf;
    char *sJ = static_cast<char *>(h->stage_J.p) + b * sj;
    const size_t w = eb * static_cast<size_t>(pc);
    if (c >= 2 && cudaStreamWaitEvent(s, h->chunk_copied[b], 0) != cudaSuccess) rc = PE_ECUDA;  // staging b free
    if (rc == PE_OK && cudaMemcpy2DAsync(spts, w, static_cast<const char *>(points) + eb * q0, hp, w, d.n,
                                         cudaMemcpyHostToDevice, s) != cudaSuccess)
      rc = PE_ECUDA;
    if (rc == PE_OK) rc = polyeval_eval(h, spts, pc, sff, sJ, stream);
    if (rc == PE_OK && (cudaEventRecord(h->chunk_done[b], s) != cudaSuccess ||
                        cudaStreamWaitEvent(h->copy_stream, h->chunk_done[b], 0) != cudaSuccess))
      rc = PE_ECUDA;
    if (rc == PE_OK && d.N > 0 &&
        (cudaMemcpy2DAsync(static_cast<char *>(out_f) + eb * q0, hp, sff, w, w, d.N, cudaMemcpyDeviceToHost,
                           h->copy_stream) != cudaSuccess ||
         cudaMemcpy2DAsync(static_cast<char *>(out_J) + eb * q0, hp, sJ, w, w, static_cast<size_t>(d.N) * d.n,
                           cudaMemcpyDeviceToHost, h->copy_stream) != cudaSuccess))
      rc = PE_ECUDA;
    if (rc == PE_OK && cudaEventRecord(h->chunk_copied[b], h->copy_stream) != cudaSuccess) rc = PE_ECUDA;
  }
  const bool ok = cudaStreamSynchronize(h->copy_stream) == cudaSuccess && cudaStreamSynchronize(s) == cudaSuccess;
  if (rc != PE_OK) return rc;
  return ok ? PE_OK : PE_ECUDA;
}

int polyeval_cost(const polyeval_t *h, double *fp64_ops, double *fp64_flops) {
  if (!h) return PE_EINVAL;
  if (fp64_ops) *fp64_ops = h->ops_per_point;
  if (fp64_flops) *fp64_flops = h->flops_per_point;
  return PE_OK;
}

int polyeval_timing(polyeval_t *h, int enable) {
  if (!h) return PE_EINVAL;
  if (enable && !h->ev[0]) {
    for (auto &e : h->ev)
      if (cudaEventCreate(&e) != cudaSuccess) return PE_ECUDA;
  }
  h->timing = enable != 0;
  h->ev_used = 0;
  h->ev_dropped = 0;
  h->kernels_launched = 0;
  return PE_OK;
}

int polyeval_timing_read(polyeval_t *h, double *total_ms, int64_t *launches, int64_t *kernels) {
  if (!h) return PE_EINVAL;
  double tot = 0.0;
  for (int i = 0; i < h->ev_used; i++) {
    if (cudaEventSynchronize(h->ev[2 * i + 1]) != cudaSuccess) return PE_ECUDA;
    float ms = 0.0f;
    if (cudaEventElapsedTime(&ms, h->ev[2 * i], h->ev[2 * i + 1]) != cudaSuccess) return PE_ECUDA;
    tot += ms;
  }
  if (total_ms) *total_ms = tot;
  if (launches) *launches = h->ev_used;
  if (kernels) *kernels = h->kernels_launched;
  h->kernels_launched = 0;
  const int dropped = h->ev_dropped;
  h->ev_used = 0;
  h->ev_dropped = 0;
  return dropped ? PE_ERANGE : PE_OK;
}

int polyeval_status(polyeval_t *h) {
  if (!h) return PE_EINVAL;
  int v = 0;
  if (cudaDeviceSynchronize() != cudaSuccess) return PE_ECUDA;
  if (cudaMemcpy(&v, h->status.p, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return PE_ECUDA;
  if (cudaMemset(h->status.p, 0, sizeof(int)) != cudaSuccess) return PE_ECUDA;
  return v ? PE_EDEVICE : PE_OK;
}

void polyeval_destroy(polyeval_t *h) { delete h; }

const char *polyeval_strerror(int code) {
  switch (code) {
    case PE_OK: return "ok";
    case PE_EINVAL: return "invalid argument or malformed system";
    case PE_ENOMEM: return "out of memory";
    case PE_ECUDA: return "CUDA runtime error";
    case PE_ERANGE: return "size beyond the limits of this build";
    case PE_EDEVICE: return "a kernel reported an inconsistent index";
    default: return "unknown status code";
  }
}

int polyeval_fp64_peak(void *stream, double *fma_per_s, double *sm_clock_mhz) {
  return pe::fp64_peak_probe(static_cast<cudaStream_t>(stream), fma_per_s, sm_clock_mhz) == cudaSuccess ? PE_OK
                                                                                                        : PE_ECUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// path tracking
// ---------------------------------------------------------------------------

namespace {

// A handle the tracker accepts: one square system in double-double or double
// whose polynomials all have degree >= 1.
bool trackable(const polyeval *h) {
  if (!h || h->batch || h->qd || h->paper) return false;
  const SysDesc &d = h->sys[0];
  if (d.N != d.n || d.n < 1 || static_cast<int32_t>(h->degrees.size()) != d.n) return false;
  for (int32_t g : h->degrees)
    if (g < 1) return false;
  return true;
}

int upload_degrees(polyeval *h) {
  if (h->deg_dev.p) return PE_OK;
  return h->deg_dev.upload(h->degrees);
}

// Scratch for tracking P paths on handle h: F, J_F, the accepted points, the
// path states and the running-path counter.
int track_scratch(polyeval *h, int64_t P) {
  const SysDesc &d = h->sys[0];
  const size_t eb = static_cast<size_t>(elem_doubles(h)) * sizeof(double);
  const size_t np = static_cast<size_t>(d.n) * static_cast<size_t>(P);
  const size_t Pz = static_cast<size_t>(P);
  int rc;
  if ((rc = upload_degrees(h)) || (rc = ensure(h->tr_f, eb * np)) || (rc = ensure(h->tr_J, eb * np * d.n)) ||
      (rc = ensure(h->tr_active, sizeof(unsigned))) || (rc = ensure(h->tr_home, sizeof(pe::TrackState) * Pz)) ||
      (rc = ensure(h->tr_list, sizeof(int64_t) * Pz)))
    return rc;
  for (int b = 0; b < 2; b++)
    if ((rc = ensure(h->tr_xw[b], eb * np)) || (rc = ensure(h->tr_xsw[b], eb * np)) ||
        (rc = ensure(h->tr_stw[b], sizeof(pe::TrackState) * Pz)) || (rc = ensure(h->tr_perm[b], sizeof(int64_t) * Pz)))
      return rc;
  return PE_OK;
}

bool params_ok(const pe_track_params *p) {
  return p && p->h_init > 0.0 && p->h_min > 0.0 && p->h_max >= p->h_init && p->h_init >= p->h_min &&
         p->corr_tol > 0.0 && p->end_tol > 0.0 && p->x_big > 0.0 && p->max_corr >= 1 && p->max_end >= 1 &&
         p->succ_grow >= 1 && p->max_iters >= 1 && std::isfinite(p->gamma_re) && std::isfinite(p->gamma_im) &&
         (p->gamma_re != 0.0 || p->gamma_im != 0.0);
}

constexpr int kGraphIters = 8;  // tracker iterations per captured graph

// Compaction: once at most half of the working batch still runs (and the
// batch has at least kCompactMin paths), every path is written home to the
// caller's array (by its original index) and the running ones are packed into
// a batch of their own, so that the long tail of slow paths no longer pays
// for evaluating the finished ones.
constexpr int64_t kCompactMin = 128;

int track(polyeval *h, const pe_track_params *prm, double *x_home, int64_t P0, double *t_out, int32_t *status,
          int64_t *iterations, cudaStream_t s) {
  if (iterations) *iterations = 0;
  if (P0 == 0) return PE_OK;
  int rc = track_scratch(h, P0);
  if (rc != PE_OK) return rc;
  const SysDesc &d = h->sys[0];
  const int words = elem_doubles(h);
  const int state_words = static_cast<int>(sizeof(pe::TrackState) / sizeof(double));
  pe::TrackParams tp{};
  tp.n = d.n;
  tp.J = static_cast<double *>(h->tr_J.p);
  tp.f = static_cast<double *>(h->tr_f.p);
  tp.deg = static_cast<const int32_t *>(h->deg_dev.p);
  tp.gre = prm->gamma_re;
  tp.gim = prm->gamma_im;
  tp.h_min = prm->h_min;
  tp.h_max = prm->h_max;
  tp.corr_tol = prm->corr_tol;
  tp.end_tol = prm->end_tol;
  tp.x_big = prm->x_big;
  tp.max_corr = prm->max_corr;
  tp.max_end = prm->max_end;
  tp.succ_grow = prm->succ_grow;
  tp.mixed = prm->mixed != 0 && h->dd;
  if (tp.mixed) {  // double copies of the systems, for warp solves outside shared memory
    const size_t np = static_cast<size_t>(d.n) * static_cast<size_t>(P0);
    if ((rc = ensure(h->tr_JL, 16 * np * d.n)) || (rc = ensure(h->tr_bL, 16 * np))) return rc;
    tp.JL = static_cast<double *>(h->tr_JL.p);
    tp.bL = static_cast<double *>(h->tr_bL.p);
  }
  tp.active = static_cast<unsigned *>(h->tr_active.p);
  // The iterations run on the handle's own stream: the batch of kGraphIters
  // iterations (counter reset, evaluation, step) is captured into a CUDA graph
  // and replayed, which removes the host overhead of its dozens of short
  // launches; the running-path count is read after each replay.
  if (!h->tr_stream && cudaStreamCreateWithFlags(&h->tr_stream, cudaStreamNonBlocking) != cudaSuccess) {
    h->tr_stream = nullptr;
    return PE_ECUDA;
  }
  cudaStream_t ts = h->tr_stream;
  if (cudaStreamSynchronize(s) != cudaSuccess) return PE_ECUDA;  // start points queued by the caller
  auto xw = [&](int b) { return static_cast<double *>(h->tr_xw[b].p); };
  auto xsw = [&](int b) { return static_cast<double *>(h->tr_xsw[b].p); };
  auto stw = [&](int b) { return static_cast<double *>(h->tr_stw[b].p); };
  auto perm = [&](int b) { return static_cast<double *>(h->tr_perm[b].p); };  // int64 bits, moved as words
  int cur = 0;
  int64_t Pc = P0;
  {  // working batch 0: the start points, paths in order
    std::vector<int64_t> iota(static_cast<size_t>(P0));
    std::iota(iota.begin(), iota.end(), int64_t{0});
    if (cudaMemcpy(perm(0), iota.data(), sizeof(int64_t) * iota.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpyAsync(xw(0), x_home, static_cast<size_t>(words) * sizeof(double) * d.n * P0,
                        cudaMemcpyDeviceToDevice, ts) != cudaSuccess)
      return PE_ECUDA;
  }
  auto bind = [&]() {
    tp.P = Pc;
    tp.x = xw(cur);
    tp.xs = xsw(cur);
    tp.st = reinterpret_cast<pe::TrackState *>(stw(cur));
  };
  bind();
  if (pe::launch_track_init(h->dd, tp, prm->h_init, ts) != cudaSuccess) return PE_ECUDA;
  const bool timing = h->timing;
  h->timing = false;  // no event pairs inside the graph
  auto iteration = [&](cudaStream_t st) -> int {
    if (cudaMemsetAsync(tp.active, 0, sizeof(unsigned), st) != cudaSuccess) return PE_ECUDA;
    int r = polyeval_eval(h, tp.x, tp.P, tp.f, tp.J, st);
    if (r != PE_OK) return r;
    if (pe::launch_track_step(h->dd, tp, st) != cudaSuccess) return PE_ECUDA;
    h->kernels_launched++;
    return PE_OK;
  };
  struct Graph {
    cudaGraph_t g = nullptr;
    cudaGraphExec_t e = nullptr;
    void reset() {
      if (e) cudaGraphExecDestroy(e);
      if (g) cudaGraphDestroy(g);
      e = nullptr;
      g = nullptr;
    }
    ~Graph() { reset(); }
  } graph;
  int64_t per_replay = 0;
  auto capture = [&]() -> int {  // a graph of kGraphIters iterations on the current batch
    graph.reset();
    if (prm->max_iters < kGraphIters) return PE_OK;
    const int64_t k0 = h->kernels_launched;
    int r = cudaStreamBeginCapture(ts, cudaStreamCaptureModeThreadLocal) == cudaSuccess ? PE_OK : PE_ECUDA;
    for (int i = 0; i < kGraphIters && r == PE_OK; i++) r = iteration(ts);
    const cudaError_t ce = cudaStreamEndCapture(ts, &graph.g);  // always leave capture mode
    if (r == PE_OK && (ce != cudaSuccess || cudaGraphInstantiate(&graph.e, graph.g, 0) != cudaSuccess)) r = PE_ECUDA;
    per_replay = h->kernels_launched - k0;
    h->kernels_launched = k0;
    if (r != PE_OK) cudaGetLastError();
    return r;
  };
  // every working path (and its state) home, by original index
  auto write_home = [&]() -> int {
    const int64_t *pm = static_cast<const int64_t *>(h->tr_perm[cur].p);
    if (pe::launch_move_paths(xw(cur), Pc, x_home, P0, pm, Pc, d.n, words, true, ts) != cudaSuccess ||
        pe::launch_move_paths(stw(cur), Pc, static_cast<double *>(h->tr_home.p), P0, pm, Pc, 1, state_words, true,
                              ts) != cudaSuccess)
      return PE_ECUDA;
    return PE_OK;
  };
  // the running paths into the other working batch
  auto compact = [&]() -> int {
    std::vector<pe::TrackState> st(static_cast<size_t>(Pc));
    if (cudaMemcpyAsync(st.data(), stw(cur), sizeof(pe::TrackState) * st.size(), cudaMemcpyDeviceToHost, ts) !=
            cudaSuccess ||
        cudaStreamSynchronize(ts) != cudaSuccess)
      return PE_ECUDA;
    std::vector<int64_t> keep;
    for (int64_t q = 0; q < Pc; q++)
      if (st[static_cast<size_t>(q)].status == pe::kPathRunning) keep.push_back(q);
    const int64_t m = static_cast<int64_t>(keep.size());
    int r = write_home();
    if (r != PE_OK || m == 0) return r;
    const int64_t *list = static_cast<const int64_t *>(h->tr_list.p);
    const int nx = 1 - cur;
    if (cudaMemcpyAsync(h->tr_list.p, keep.data(), sizeof(int64_t) * keep.size(), cudaMemcpyHostToDevice, ts) !=
            cudaSuccess ||
        pe::launch_move_paths(xw(cur), Pc, xw(nx), m, list, m, d.n, words, false, ts) != cudaSuccess ||
        pe::launch_move_paths(xsw(cur), Pc, xsw(nx), m, list, m, d.n, words, false, ts) != cudaSuccess ||
        pe::launch_move_paths(stw(cur), Pc, stw(nx), m, list, m, 1, state_words, false, ts) != cudaSuccess ||
        pe::launch_move_paths(perm(cur), Pc, perm(nx), m, list, m, 1, 1, false, ts) != cudaSuccess ||
        cudaStreamSynchronize(ts) != cudaSuccess)  // `keep` is read by the copy
      return PE_ECUDA;
    cur = nx;
    Pc = m;
    bind();
    return capture();
  };
  rc = capture();
  int64_t it = 0;
  unsigned running = 1;
  while (rc == PE_OK && it < prm->max_iters && running) {
    if (graph.e && it + kGraphIters <= prm->max_iters) {
      if (cudaGraphLaunch(graph.e, ts) != cudaSuccess) rc = PE_ECUDA;
      h->kernels_launched += per_replay;
      it += kGraphIters;
    } else {
      rc = iteration(ts);
      it++;
    }
    if (rc == PE_OK && (cudaMemcpyAsync(&running, tp.active, sizeof(unsigned), cudaMemcpyDeviceToHost, ts) !=
                            cudaSuccess ||
                        cudaStreamSynchronize(ts) != cudaSuccess))
      rc = PE_ECUDA;
    if (rc == PE_OK && running && Pc >= kCompactMin && 2 * static_cast<int64_t>(running) <= Pc) rc = compact();
  }
  h->timing = timing;
  if (rc == PE_OK) rc = write_home();
  if (rc != PE_OK) return rc;
  if (pe::launch_track_finish(static_cast<const pe::TrackState *>(h->tr_home.p), P0, t_out, status, ts) !=
      cudaSuccess)
    return PE_ECUDA;
  if (iterations) *iterations = it;
  return cudaStreamSynchronize(ts) == cudaSuccess ? PE_OK : PE_ECUDA;
}

}  // namespace

extern "C" {

int polyeval_track_defaults(int precision, pe_track_params *prm) {
  if (!prm || !valid_precision(precision) || precision == PE_QD_INT) return PE_EINVAL;
  const bool dd = precision != PE_F64;
  prm->gamma_re = 0.5403023058681398;  // exp(i): a fixed point of the unit circle off every axis
  prm->gamma_im = 0.8414709848078965;
  prm->h_init = 0.02;
  prm->h_min = dd ? 1e-14 : 1e-10;
  prm->h_max = 0.1;
  // Path following needs only to stay on the path; the end point is refined
  // to end_tol at t = 1.  A corrector tolerance of 1e-6 took 40 % of the
  // iterations of 1e-9 on generic dense systems with every end point
  // distinct, and kept paths that go to infinity from jumping onto finite
  // roots; allowing a fourth corrector step (or larger h_max) let paths jump.
  prm->corr_tol = 1e-6;
  prm->end_tol = dd ? 1e-26 : 1e-13;
  prm->x_big = 1e8;
  prm->max_corr = 3;
  prm->max_end = 8;
  prm->succ_grow = 3;
  prm->mixed = dd ? 1 : 0;
  prm->max_iters = 100000;
  return PE_OK;
}

int polyeval_bezout(const polyeval_t *h, double *count, int32_t *degrees) {
  if (!h || h->batch || h->degrees.empty()) return PE_EINVAL;
  double c = 1.0;
  for (size_t i = 0; i < h->degrees.size(); i++) {
    c *= h->degrees[i];
    if (degrees) degrees[i] = h->degrees[i];
  }
  if (count) *count = c;
  return PE_OK;
}

int polyeval_start_points(polyeval_t *h, int64_t first, int64_t P, void *points, void *stream) {
  if (!trackable(h) || first < 0 || P < 0) return PE_EINVAL;
  if (P == 0) return PE_OK;
  if (!points || !aligned16(points)) return PE_EINVAL;
  int rc;
  if ((rc = upload_degrees(h)) != PE_OK) return rc;
  return pe::launch_start_points(h->dd, h->sys[0].n, static_cast<const int32_t *>(h->deg_dev.p), first, P,
                                 static_cast<double *>(points), static_cast<cudaStream_t>(stream)) == cudaSuccess
             ? PE_OK
             : PE_ECUDA;
}

int polyeval_track(polyeval_t *h, const pe_track_params *prm, void *points, int64_t P, double *t, int32_t *status,
                   int64_t *iterations, void *stream) {
  if (iterations) *iterations = 0;
  if (!trackable(h) || !params_ok(prm) || P < 0) return PE_EINVAL;
  if (P > h->max_points) return PE_ERANGE;
  if (P > 0 && (!points || !aligned16(points))) return PE_EINVAL;
  return track(h, prm, static_cast<double *>(points), P, t, status, iterations, static_cast<cudaStream_t>(stream));
}

int polyeval_track_adaptive(polyeval_t *h_lo, polyeval_t *h_hi, const pe_track_params *prm_lo,
                            const pe_track_params *prm_hi, void *points, int64_t P, int32_t *status,
                            int64_t *escalated, void *stream) {
  if (escalated) *escalated = 0;
  if (!trackable(h_lo) || !trackable(h_hi) || h_lo->dd || !h_hi->dd || !params_ok(prm_lo) || !params_ok(prm_hi) ||
      P < 0)
    return PE_EINVAL;
  if (h_lo->sys[0].n != h_hi->sys[0].n || h_lo->degrees != h_hi->degrees) return PE_EINVAL;
  if (P > h_lo->max_points || P > h_hi->max_points) return PE_ERANGE;
  if (P == 0) return PE_OK;
  if (!points || !status || !aligned16(points)) return PE_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int32_t n = h_hi->sys[0].n;
  double *x = static_cast<double *>(points);
  const int64_t count = static_cast<int64_t>(n) * P;
  int rc;
  if ((rc = ensure(h_lo->tr_x64, sizeof(double) * 2 * static_cast<size_t>(count))) ||
      (rc = ensure(h_lo->tr_status, sizeof(int32_t) * static_cast<size_t>(P))) || (rc = track_scratch(h_hi, P)))
    return rc;
  double *x64 = static_cast<double *>(h_lo->tr_x64.p);
  int32_t *st_lo = static_cast<int32_t *>(h_lo->tr_status.p);
  // 1. every path in double precision
  if (pe::launch_narrow_points(x, x64, count, s) != cudaSuccess) return PE_ECUDA;
  if ((rc = track(h_lo, prm_lo, x64, P, nullptr, st_lo, nullptr, s)) != PE_OK) return rc;
  std::vector<int32_t> st(static_cast<size_t>(P));
  if (cudaMemcpy(st.data(), st_lo, sizeof(int32_t) * st.size(), cudaMemcpyDeviceToHost) != cudaSuccess)
    return PE_ECUDA;
  std::vector<int64_t> redo;
  for (int64_t q = 0; q < P; q++)
    if (st[static_cast<size_t>(q)] != pe::kPathSuccess) redo.push_back(q);
  const int64_t m = static_cast<int64_t>(redo.size());
  // 2. the start points of the paths that did not succeed, set aside
  if (m > 0) {
    if ((rc = ensure(h_hi->tr_xc, sizeof(double) * 4 * static_cast<size_t>(n) * m)) ||
        (rc = ensure(h_hi->tr_statc, sizeof(int32_t) * static_cast<size_t>(m))) ||
        (rc = ensure(h_hi->tr_idx, sizeof(int64_t) * static_cast<size_t>(m))))
      return rc;
    if (cudaMemcpyAsync(h_hi->tr_idx.p, redo.data(), sizeof(int64_t) * redo.size(), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
      return PE_ECUDA;
    if (pe::launch_move_paths(x, P, static_cast<double *>(h_hi->tr_xc.p), m, static_cast<const int64_t *>(h_hi->tr_idx.p),
                              m, n, 4, false, s) != cudaSuccess)
      return PE_ECUDA;
  }
  // 3. the double-precision endpoints, refined by Newton's method in double-double
  if (pe::launch_widen_points(x64, x, count, s) != cudaSuccess) return PE_ECUDA;
  for (int k = 0; k < 3; k++)
    if ((rc = polyeval_newton(h_hi, x, P, h_hi->tr_f.p, h_hi->tr_J.p, nullptr, s)) != PE_OK) return rc;
  if (cudaMemcpyAsync(status, st_lo, sizeof(int32_t) * static_cast<size_t>(P), cudaMemcpyDeviceToDevice, s) !=
      cudaSuccess)
    return PE_ECUDA;
  // 4. the others tracked again from their start points in double-double
  if (m > 0) {
    if (m > h_hi->max_points) return PE_ERANGE;
    double *xc = static_cast<double *>(h_hi->tr_xc.p);
    int32_t *stc = static_cast<int32_t *>(h_hi->tr_statc.p);
    pe_track_params full = *prm_hi;
    full.mixed = 0;
    if ((rc = track(h_hi, &full, xc, m, nullptr, stc, nullptr, s)) != PE_OK) return rc;
    const int64_t *idx = static_cast<const int64_t *>(h_hi->tr_idx.p);
    if (pe::launch_move_paths(xc, m, x, P, idx, m, n, 4, true, s) != cudaSuccess ||
        pe::launch_scatter_status(stc, status, idx, m, s) != cudaSuccess)
      return PE_ECUDA;
  }
  if (escalated) *escalated = m;
  return cudaStreamSynchronize(s) == cudaSuccess ? PE_OK : PE_ECUDA;
}

}  // extern "C"
