// Decoding of a work item of the main kernels (kernels.cu, kernels_wide.cu).
//
// A single-system call has T x N x C items: tile of 16 points, polynomial
// rank r (in decreasing cost order within the tile), and chunk of the
// polynomial's monomials (C = 1 unless the call has too few (polynomial,
// tile) pairs to fill the GPU).  Tile-major order keeps the warps that run at
// the same time on few tiles, so their points and power-table entries are
// read from L2 rather than DRAM (n = 128, k = 32: 5 % less DRAM traffic in
// double-double, 3 % faster with integer-pipe products).  Chunk 0 writes f and J into the outputs; chunk c > 0 into scratch
// copy c-1 of the same layout, which a combine kernel adds afterwards.  A
// batch handle has C items per (polynomial, tile) entry of its item table,
// chunked the same way.
#pragma once

#include <cstdint>

#include "internal.h"

namespace pe {

struct Item {
  int gp, tile, s, P;  // global polynomial, tile (of 16 / groups points), system, points of the system
  int groups;          // monomial groups per warp
  int t0, t1;          // monomial range
  double *f_base;      // output (or scratch) base for f
  double *J_base;      // output (or scratch) base for J
};

// Returns false (and flags the status word) for an inconsistent item.
__device__ __forceinline__ bool decode_item(const MainParams &kp, unsigned item, int lane, Item &it) {
  int chunk = 0;
  if (kp.single_P >= 0) {
    const unsigned C = static_cast<unsigned>(kp.n_chunks);
    const unsigned rest = item / C;
    chunk = static_cast<int>(item - rest * C);
    it.tile = static_cast<int>(rest) / kp.n_polys_total;  // tile-major: the warps resident at once share tiles
    const int r = static_cast<int>(rest) - it.tile * kp.n_polys_total;
    it.gp = kp.perm[r];
    it.s = 0;
    it.P = kp.single_P;
    it.groups = kp.groups;
  } else {
    const unsigned C = static_cast<unsigned>(kp.n_chunks);
    const unsigned rest = item / C;
    chunk = static_cast<int>(item - rest * C);
    const int2 x = kp.items[rest];
    it.gp = x.x;
    it.groups = 1 << ((x.y >> kTileBits) & 7);
    it.tile = (x.y & ((1 << kTileBits) - 1)) * it.groups;  // in tiles of 16 / groups points
    it.s = (x.x >= 0 && x.x < kp.n_polys_total) ? kp.poly_sys[x.x] : 0;
    it.P = kp.sys[it.s].P;
  }
  if (it.gp < 0 || it.gp >= kp.n_polys_total || it.groups > kPointsPerWarp ||
      it.tile * (kPointsPerWarp / it.groups) >= it.P) {
    if (lane == 0) atomicOr(kp.status, 1);
    return false;
  }
  int t0 = kp.poly_ptr[it.gp], t1 = kp.poly_ptr[it.gp + 1];
  if (kp.n_chunks > 1) {
    const long long m = t1 - t0;
    const int a = t0 + static_cast<int>(m * chunk / kp.n_chunks);
    const int b = t0 + static_cast<int>(m * (chunk + 1) / kp.n_chunks);
    t0 = a;
    t1 = b;
  }
  it.t0 = t0;
  it.t1 = t1;
  it.f_base = chunk == 0 ? kp.out_f : kp.scratch_f + static_cast<size_t>(chunk - 1) * kp.chunk_f_stride;
  it.J_base = chunk == 0 ? kp.out_J : kp.scratch_J + static_cast<size_t>(chunk - 1) * kp.chunk_J_stride;
  return true;
}

}  // namespace pe
