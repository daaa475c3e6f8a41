// polyeval_eval_noalloc: evaluation of f and J for callers that cannot
// allocate device memory.
//
// Who needs it: code whose device memory is owned by someone else -- a
// framework's caching allocator, a pre-reserved arena of a real-time or
// embedded application, or a host program whose memory budget is fixed once
// at start-up -- cannot let this library call cudaMalloc, and so cannot use
// polyeval_create, which copies the system into device memory it allocates
// and keeps a power table sized for the largest batch.  Such a caller places
// the system arrays, the points and the outputs in its own device memory and
// calls this entry point, which allocates nothing.
//
// The only scratch the evaluation needs, the table of powers x^2 .. x^(d-1)
// of every variable at every point, lives in the file-scope device array
// below.  It is a fixed kNoAllocScratchBytes (16 MiB) that every GPU which
// loads this library holds until the process exits.  Every call uses the same
// array: each call writes every table entry it reads before reading it (in
// stream order), so nothing in it has to start at zero, but two calls whose
// kernels overlap on the GPU (different streams, or different host threads)
// race on it and give wrong results.
//
// This is the same evaluation as polyeval_create + polyeval_eval in complex
// double-double (one warp per polynomial and tile of 16 points, lane pairs
// holding real and imaginary parts); it reads the system in the plain
// compressed-row format of pe_system instead of the compiled one.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "dd.cuh"
#include "internal.h"
#include "polyeval.h"

namespace pe {
namespace noalloc {

constexpr size_t kNoAllocScratchBytes = size_t{16} << 20;
constexpr int kMaxK = 256;  // prefix-product slots per warp: (kMaxK - 1) * 512 bytes of shared memory
constexpr int kTile = 16;
constexpr int kMaxDevices = 64;
constexpr unsigned long long kSignBit = 0x8000000000000000ULL;

static __device__ __align__(256) unsigned char pe_noalloc_scratch[kNoAllocScratchBytes];

struct Params {
  int32_t n, N, max_k, max_exp, P, T;
  const int64_t *poly_ptr;
  const int64_t *mono_ptr;
  const int32_t *pos;
  const int32_t *exps;
  const double *coef;
  const double *points;
  double *out_f;
  double *out_J;
  double *table;
};

struct Cdd {
  dd re, im;
};

__device__ __forceinline__ Cdd load_cdd(const double *p) {
  const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
  const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
  return Cdd{dd{a.x, a.y}, dd{b.x, b.y}};
}

__device__ __forceinline__ Cdd load_cdd_coherent(const double *p) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0];
  const double2 b = reinterpret_cast<const double2 *>(p)[1];
  return Cdd{dd{a.x, a.y}, dd{b.x, b.y}};
}

// y (split over the lane pair) times X (full complex value on both lanes).
__device__ __forceinline__ dd mul_by(dd y, const Cdd &X, unsigned long long sgn, bool norm) {
  const dd yp = shfl_xor(y, 1);
  const dd a2 = negate_if(X.im, sgn);
  return norm ? dot2n(X.re, y, a2, yp) : dot2(X.re, y, a2, yp);
}

// P * Q, both split over the lane pair (final product, not renormalised).
__device__ __forceinline__ dd mul_pair(dd P, dd Q, int c, unsigned long long sgn) {
  const dd Pp = shfl_xor(P, 1), Qp = shfl_xor(Q, 1);
  const bool re = c == 0;
  return dot2(P, select(re, Q, Qp), negate_if(Pp, sgn), select(re, Qp, Q));
}

__global__ void powers(const Params p) {
  const int64_t total = static_cast<int64_t>(p.n) * p.P;
  const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
  for (int64_t idx = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const int64_t v = idx / p.P, q = idx - v * p.P;
    const Cdd x = load_cdd(p.points + (v * p.P + q) * 4);
    auto entry = [&](int e) { return p.table + ((static_cast<int64_t>(e - 2) * p.n + v) * p.P + q) * 4; };
    for (int e = 2; e < p.max_exp; e++) {
      const int h = e >> 1, g = e - h;
      const Cdd lo = h == 1 ? x : load_cdd_coherent(entry(h));
      const Cdd hi = g == 1 ? x : load_cdd_coherent(entry(g));
      const Cdd z{dot2n(hi.re, lo.re, negate_if(hi.im, kSignBit), lo.im), dot2n(hi.re, lo.im, hi.im, lo.re)};
      double *d = entry(e);
      reinterpret_cast<double2 *>(d)[0] = make_double2(z.re.h, z.re.l);
      reinterpret_cast<double2 *>(d)[1] = make_double2(z.im.h, z.im.l);
    }
  }
}

// One warp per (polynomial, tile of 16 points).  Metadata that breaks the
// stated limits (k > max_k, exponent outside 1..max_exp, position outside
// 0..n-1) is never dereferenced: the monomial is skipped and f of that
// polynomial is written as NaN so the caller sees it.
__global__ void __launch_bounds__(32) evaluate(const Params p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  dd *slots = reinterpret_cast<dd *>(smem_raw);
  const int lane = threadIdx.x & 31;
  const int64_t item = blockIdx.x;
  const int poly = static_cast<int>(item / p.T), tile = static_cast<int>(item - static_cast<int64_t>(poly) * p.T);
  const int q = tile * kTile + (lane >> 1);
  const bool valid = q < p.P;
  const int qc = valid ? q : p.P - 1;
  const int c = lane & 1;
  const unsigned long long sgn = c ? 0ULL : kSignBit;
  const size_t P = static_cast<size_t>(p.P);
  double *Jrow = p.out_J + static_cast<size_t>(poly) * p.n * P * 4;
  auto xel = [&](int v) { return p.points + (static_cast<size_t>(v) * P + qc) * 4; };
  auto tel = [&](int e, int v) { return p.table + ((static_cast<size_t>(e - 2) * p.n + v) * P + qc) * 4; };
  auto jel = [&](int v) { return Jrow + (static_cast<size_t>(v) * P + qc) * 4; };

  if (valid)
    for (int v = 0; v < p.n; v++) reinterpret_cast<double2 *>(jel(v))[c] = make_double2(0.0, 0.0);
  dd f{0.0, 0.0};
  bool bad = false;
  const int64_t t0 = p.poly_ptr[poly], t1 = p.poly_ptr[poly + 1];
  for (int64_t t = t0; t < t1; t++) {
    const int64_t vb = p.mono_ptr[t];
    const int64_t kk = p.mono_ptr[t + 1] - vb;
    bool ok = kk >= 0 && kk <= p.max_k;
    for (int64_t j = 0; ok && j < kk; j++) {
      const int v = __ldg(p.pos + vb + j), a = __ldg(p.exps + vb + j);
      ok = v >= 0 && v < p.n && a >= 1 && a <= p.max_exp;
    }
    if (!ok) {
      bad = true;
      continue;
    }
    const int k = static_cast<int>(kk);
    const double2 cw = __ldg(reinterpret_cast<const double2 *>(p.coef + static_cast<size_t>(t) * 4) + c);
    dd G{cw.x, cw.y};
    if (k == 0) {
      f = add(f, G);
      continue;
    }
    const int32_t *pv = p.pos + vb;
    const int32_t *pa = p.exps + vb;
    for (int j = 0; j < k; j++) {
      const int v = __ldg(pv + j), a = __ldg(pa + j);
      if (a >= 2) G = mul_by(G, load_cdd(a == 2 ? xel(v) : tel(a - 1, v)), sgn, true);
    }
    dd Pc = G;
    for (int j = 0; j < k - 1; j++) {
      slots[j * 32 + lane] = Pc;
      Pc = mul_by(Pc, load_cdd(xel(__ldg(pv + j))), sgn, true);
    }
    const int vl = __ldg(pv + k - 1), al = __ldg(pa + k - 1);
    const Cdd xl = load_cdd(xel(vl));
    f = add(f, mul_by(Pc, xl, sgn, false));
    {
      const dd d = al == 1 ? Pc : scale(Pc, int_as_double(al));
      double2 *acc = reinterpret_cast<double2 *>(jel(vl)) + c;
      const double2 o = *acc;
      const dd s = add(dd{o.x, o.y}, d);
      if (valid) *acc = make_double2(s.h, s.l);
    }
    dd Q = select(c == 0, xl.re, xl.im);
    for (int j = k - 2; j >= 0; j--) {
      const int v = __ldg(pv + j), a = __ldg(pa + j);
      const dd D = mul_pair(slots[j * 32 + lane], Q, c, sgn);
      const dd d = a == 1 ? D : scale(D, int_as_double(a));
      double2 *acc = reinterpret_cast<double2 *>(jel(v)) + c;
      const double2 o = *acc;
      const dd s = add(dd{o.x, o.y}, d);
      if (valid) *acc = make_double2(s.h, s.l);
      if (j > 0) Q = mul_by(Q, load_cdd(xel(v)), sgn, true);
    }
  }
  if (valid) {
    const dd fo = bad ? dd{__longlong_as_double(0x7ff8000000000000LL), 0.0} : normalize(f);
    reinterpret_cast<double2 *>(p.out_f + (static_cast<size_t>(poly) * P + q) * 4)[c] = make_double2(fo.h, fo.l);
    for (int v = 0; v < p.n; v++) {
      double2 *acc = reinterpret_cast<double2 *>(jel(v)) + c;
      const double2 o = *acc;
      const dd s = normalize(dd{o.x, o.y});
      *acc = make_double2(s.h, s.l);
    }
  }
}

// Device address of the scratch array, looked up once per device.
std::mutex g_setup_mutex;
void *g_scratch[kMaxDevices] = {};

int setup(int dev, void **scratch) {
  if (dev < 0 || dev >= kMaxDevices) return PE_ERANGE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, pe_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();
      return PE_ECUDA;
    }
    int optin = 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return PE_ECUDA;
    if (cudaFuncSetAttribute(evaluate, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) != cudaSuccess)
      return PE_ECUDA;
    g_scratch[dev] = ptr;
  }
  *scratch = g_scratch[dev];
  return PE_OK;
}

}  // namespace noalloc
}  // namespace pe

extern "C" PE_API int polyeval_eval_noalloc(const pe_system *dev_sys, int32_t max_k, int32_t max_exp,
                                            const void *points, int64_t P, void *out_f, void *out_J, void *stream) {
  using namespace pe::noalloc;
  if (!dev_sys || P < 0 || max_k < 0 || max_exp < 1) return PE_EINVAL;
  if (dev_sys->n_vars < 1 || dev_sys->n_polys < 0) return PE_EINVAL;
  if (dev_sys->n_vars > PE_MAX_VARS || max_exp > PE_MAX_EXP || max_k > kMaxK || P > INT32_MAX) return PE_ERANGE;
  if (P == 0 || dev_sys->n_polys == 0) return PE_OK;
  if (!dev_sys->poly_ptr || !dev_sys->mono_ptr || !dev_sys->pos || !dev_sys->exp || !dev_sys->coef || !points ||
      !out_f || !out_J)
    return PE_EINVAL;
  // 16-byte vector accesses of points, coefficients and outputs
  const auto misaligned = [](const void *q) { return (reinterpret_cast<uintptr_t>(q) & 15u) != 0; };
  if (misaligned(points) || misaligned(out_f) || misaligned(out_J) || misaligned(dev_sys->coef)) return PE_EINVAL;
  const int64_t table_entries = max_exp > 2 ? static_cast<int64_t>(max_exp - 2) * dev_sys->n_vars * P : 0;
  if (table_entries > static_cast<int64_t>(kNoAllocScratchBytes / (4 * sizeof(double)))) return PE_ERANGE;
  const int64_t T = (P + kTile - 1) / kTile;
  const int64_t items = static_cast<int64_t>(dev_sys->n_polys) * T;
  if (items > INT32_MAX) return PE_ERANGE;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return PE_ECUDA;
  void *scratch = nullptr;
  const int rc = setup(dev, &scratch);
  if (rc != PE_OK) return rc;

  Params p{};
  p.n = dev_sys->n_vars;
  p.N = dev_sys->n_polys;
  p.max_k = max_k;
  p.max_exp = max_exp;
  p.P = static_cast<int32_t>(P);
  p.T = static_cast<int32_t>(T);
  p.poly_ptr = dev_sys->poly_ptr;
  p.mono_ptr = dev_sys->mono_ptr;
  p.pos = dev_sys->pos;
  p.exps = dev_sys->exp;
  p.coef = reinterpret_cast<const double *>(dev_sys->coef);
  p.points = static_cast<const double *>(points);
  p.out_f = static_cast<double *>(out_f);
  p.out_J = static_cast<double *>(out_J);
  p.table = static_cast<double *>(scratch);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (max_exp > 2) {
    const int64_t total = static_cast<int64_t>(p.n) * P;
    int64_t blocks = (total + 255) / 256;
    if (blocks > pe::kSms * 64) blocks = pe::kSms * 64;
    powers<<<static_cast<unsigned>(blocks), 256, 0, s>>>(p);
    if (cudaGetLastError() != cudaSuccess) return PE_ECUDA;
  }
  const size_t smem = static_cast<size_t>(max_k > 1 ? max_k - 1 : 1) * 32 * sizeof(pe::dd);
  evaluate<<<static_cast<unsigned>(items), 32, smem, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? PE_OK : PE_ECUDA;
}
