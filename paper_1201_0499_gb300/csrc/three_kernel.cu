// The paper's own three-kernel design, for comparison with the fused kernel
// (create flag PE_PAPER_KERNELS).  Complex double-double, regular systems
// (every polynomial m monomials, every monomial k >= 3 variables), one
// thread per monomial as in Sections 3.1-3.3, batched over points with the
// point as the second grid dimension:
//
//  K1 (Section 3.1): each block of 32 threads first computes, with its first
//     n threads, the powers x^2 .. x^(d-1) of every variable into shared
//     memory (every block its own table), then each thread multiplies the k
//     factors x^(a-1) of its monomial (k - 1 products) and writes the common
//     factor to global memory, coalesced.
//  K2 (Section 3.2): each thread evaluates the Speelpenning product of its
//     monomial and all its derivatives with forward products in shared
//     locations L_2 .. L_k and one backward product Q (3k - 6 products),
//     multiplies them by the common factor (k), forms the monomial value (1)
//     and multiplies value and derivatives by their coefficients from the
//     derivative-major Coeffs array (k + 1; 5k - 4 in all), and scatters the
//     k + 1 terms into Mons.
//  K3 (Section 3.3): one thread per output (n values of f and n^2 entries of
//     J) adds exactly m terms of Mons, zero terms included; Mons is
//     term-major, so the reads of a warp are coalesced.
//
// Mons has (n^2 + n) m entries per point, zeroed once at create; K2 writes
// only the n m (k + 1) nonzero ones.
#include <cuda_runtime.h>

#include <cstdint>

#include "cplx.cuh"
#include "dd.cuh"
#include "internal.h"

namespace pe {

constexpr int kPaperBlock = 32;  // threads per block in all three kernels (Section 4)

__device__ __forceinline__ CDD one_cdd() { return CDD{dd{1.0, 0.0}, dd{0.0, 0.0}}; }

__global__ void paper_k1(const PaperParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CDD *powers = reinterpret_cast<CDD *>(smem_raw);  // [e-1][v], e = 1 .. d-1
  const int q = blockIdx.y;
  const size_t P = static_cast<size_t>(p.P);
  const int levels = p.d - 1 > 0 ? p.d - 1 : 1;
  for (int v = threadIdx.x; v < p.n; v += blockDim.x) {
    const CDD x = CDD::load(p.points + (static_cast<size_t>(v) * P + q) * 4);
    powers[v] = x;
    CDD pw = x;
    for (int e = 2; e <= p.d - 1; e++) {  // powers 2 .. d-1, one product each
      pw = CDD::mul(pw, x);
      powers[static_cast<size_t>(e - 1) * p.n + v] = pw;
    }
  }
  (void)levels;
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.M) return;
  const uint32_t *w = p.var + static_cast<size_t>(t) * p.k;
  auto factor = [&](int j) {
    const int v = static_cast<int>(w[j] & 0xffffu), a = static_cast<int>(w[j] >> 16);
    return a == 1 ? one_cdd() : powers[static_cast<size_t>(a - 2) * p.n + v];
  };
  CDD cf = factor(0);
  for (int j = 1; j < p.k; j++) cf = CDD::mul(cf, factor(j));  // k - 1 products
  cf.store(p.cf + (static_cast<size_t>(q) * p.M + t) * 4);
}

__global__ void paper_k2(const PaperParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  CDD *xs = reinterpret_cast<CDD *>(smem_raw);  // [n]
  CDD *L = xs + p.n;                            // [k + 1][blockDim.x]
  const int q = blockIdx.y;
  const size_t P = static_cast<size_t>(p.P);
  for (int v = threadIdx.x; v < p.n; v += blockDim.x) xs[v] = CDD::load(p.points + (static_cast<size_t>(v) * P + q) * 4);
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.M) return;
  const int k = p.k, tid = threadIdx.x, B = blockDim.x;
  const uint32_t *w = p.var + static_cast<size_t>(t) * k;
  auto X = [&](int j) { return xs[w[j] & 0xffffu]; };     // x_{i_{j+1}}, j 0-based
  auto Ls = [&](int j) -> CDD & { return L[static_cast<size_t>(j) * B + tid]; };  // L_j, j 1-based
  // forward products: L_2 = x_{i1}, L_{r+2} = x_{i1} ... x_{i(r+1)}, r = 1 .. k-2
  Ls(2) = X(0);
  for (int r = 1; r <= k - 2; r++) Ls(r + 2) = CDD::mul(Ls(r + 1), X(r));
  // backward: Q = x_{ik}; L_{k-1} *= Q; then Q *= x_{i(k-r)}, L_{k-r-1} *= Q
  CDD Q = X(k - 1);
  Ls(k - 1) = CDD::mul(Ls(k - 1), Q);
  for (int r = 1; r <= k - 3; r++) {
    Q = CDD::mul(Q, X(k - 1 - r));
    Ls(k - r - 1) = CDD::mul(Ls(k - r - 1), Q);
  }
  Ls(1) = CDD::mul(Q, X(1));  // derivative by x_{i1}
  // monomial derivatives (times the common factor), value, coefficients
  const CDD cf = CDD::load(p.cf + (static_cast<size_t>(q) * p.M + t) * 4);
  for (int j = 1; j <= k; j++) Ls(j) = CDD::mul(Ls(j), cf);
  Ls(k + 1) = CDD::mul(Ls(k), X(k - 1));
  const size_t nm = static_cast<size_t>(p.M);
  for (int j = 1; j <= k + 1; j++) Ls(j) = CDD::mul(Ls(j), CDD::load(p.coeffs + ((j - 1) * nm + t) * 4));
  // scatter into Mons: value of polynomial pp at slot pp, derivative by x_i at n_polys + i n_polys + pp
  const int pp = t / p.m, tl = t - pp * p.m;
  const size_t slots = static_cast<size_t>(p.N) * (p.n + 1);
  double *row = p.mons + (static_cast<size_t>(q) * p.m + tl) * slots * 4;
  Ls(k + 1).store(row + static_cast<size_t>(pp) * 4);
  for (int j = 1; j <= k; j++) {
    const int i = static_cast<int>(w[j - 1] & 0xffffu);
    Ls(j).store(row + (static_cast<size_t>(p.N) + static_cast<size_t>(i) * p.N + pp) * 4);
  }
}

__global__ void paper_k3(const PaperParams p) {
  const int q = blockIdx.y;
  const size_t slots = static_cast<size_t>(p.N) * (p.n + 1);
  const size_t s = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= slots) return;
  const double *base = p.mons + static_cast<size_t>(q) * p.m * slots * 4;
  CDD acc = CDD::zero();
  for (int j = 0; j < p.m; j++) acc = CDD::add2(acc, CDD::load(base + (static_cast<size_t>(j) * slots + s) * 4));
  acc = acc.finish();
  const size_t P = static_cast<size_t>(p.P);
  if (s < static_cast<size_t>(p.N)) {
    acc.store(p.out_f + (s * P + q) * 4);
  } else {
    const size_t r = s - p.N, i = r / p.N, pp = r - i * p.N;
    acc.store(p.out_J + ((pp * p.n + i) * P + q) * 4);
  }
}

cudaError_t launch_paper(const PaperParams &p, cudaStream_t s) {
  if (p.P <= 0 || p.M <= 0) return cudaSuccess;
  const dim3 g12((p.M + kPaperBlock - 1) / kPaperBlock, static_cast<unsigned>(p.P));
  const size_t sm1 = sizeof(CDD) * static_cast<size_t>(p.n) * (p.d > 2 ? p.d - 1 : 1);
  const size_t sm2 = sizeof(CDD) * (static_cast<size_t>(p.n) + static_cast<size_t>(p.k + 2) * kPaperBlock);
  paper_k1<<<g12, kPaperBlock, sm1, s>>>(p);
  paper_k2<<<g12, kPaperBlock, sm2, s>>>(p);
  const size_t slots = static_cast<size_t>(p.N) * (p.n + 1);
  const dim3 g3(static_cast<unsigned>((slots + kPaperBlock - 1) / kPaperBlock), static_cast<unsigned>(p.P));
  paper_k3<<<g3, kPaperBlock, 0, s>>>(p);
  return cudaGetLastError();
}

cudaError_t prepare_paper(size_t smem_k1, size_t smem_k2) {
  cudaError_t e = cudaFuncSetAttribute(paper_k1, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_k1));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(paper_k2, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem_k2));
}

}  // namespace pe
