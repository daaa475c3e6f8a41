// Internal interface between the host side (host.cpp) and the kernels
// (kernels.cu).  Not part of the public C ABI.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace pe {

// Points handled by one warp: two lanes per point, lane 2q holds the real
// part and lane 2q+1 the imaginary part of every value of point q.
constexpr int kPointsPerWarp = 16;
constexpr int kWarpsPerBlockMax = 4;
// A batch item's tile word: the 16-point tile index in bits 0..26 and log2 of
// its monomial groups per warp in bits 27..29 (groups > 1 for the last,
// partial tile of a system with double-double or double arithmetic).
constexpr int kTileBits = 27;
// A product that feeds another product in a chain (common factor, forward
// and backward products) is renormalised every kChainRenorm-th step only.
// Left unnormalised, a complex double-double product's low word grows by at
// most about 2.5 u of the product per step (the rounding of the high word,
// the two exact product errors and the cross terms with the operands' low
// words), so r steps after a renormalisation it is within about 2.5 r u.
// What a product then drops -- the product of the low words (the factor read
// from memory is normalised, so below 2.5 r u * u / 2) and the six roundings
// of the low-word sums (each below u / 2 of a sum of at most 2.5 (r + 1) u) --
// is of order 10 r u^2.  With r = 4 a chain of 85 products (k = 32, 24
// exponents >= 2) stays within about 3e-29 of its value even if every error
// has the same sign.  A renormalisation costs 3 FP64 instructions against 13
// for the product, so every fourth step instead of every second saves about
// 4 % of the evaluation's FP64 instructions.
constexpr int kChainRenorm = 4;

// Streaming-multiprocessor count of a GB300 (two dies of 76): the grids of
// the grid-stride kernels are capped at a whole number of blocks per SM.
// Launches whose balance depends on it query the device instead.
constexpr int kSms = 152;

// One compiled system inside a handle.  Offsets are in complex elements of
// the handle's precision.
struct SysDesc {
  int32_t n;       // variables
  int32_t N;       // polynomials
  int32_t emax;    // largest exponent
  int32_t P;       // points (batch handles; single handles pass P per call)
  int32_t poly0;   // first global polynomial index
  int32_t tiles;   // ceil(P / kPointsPerWarp) (batch handles)
  int64_t pt_off;  // points  [n][P]
  int64_t f_off;   // f       [N][P]
  int64_t J_off;   // J       [N][n][P]
  int64_t tab_off; // powers  [emax-2][n][P]  (x^2 .. x^(emax-1))
};

struct MainParams {
  const int32_t *poly_ptr;  // [Ntot+1] global monomial offsets
  const int32_t *mono_ptr;  // [Mtot+1] offsets into var
  const uint32_t *var;      // [nnz] position | exponent << 16
  const double *coef;       // [Mtot] complex coefficients (4 or 2 doubles; block format for the integer paths)
  const int32_t *poly_sys;  // [Ntot] system of each global polynomial
  const SysDesc *sys;       // [count]
  const int32_t *perm;      // single handle: polynomials by decreasing cost
  const int2 *items;        // batch handle: (global polynomial, tile) by decreasing cost
  const double *points;
  double *out_f;
  double *out_J;
  const double *table;
  int64_t n_items;
  int32_t single_P;         // >= 0: single-system handle evaluated at single_P points
  int32_t single_T;         // tiles of a single-system call
  int32_t tile_points;      // points per tile: kPointsPerWarp / groups
  int32_t groups;           // monomial groups per warp (1, 2, 4, 8, 16; double-double and double only)
  int32_t kslots;           // prefix-product slots per lane (max k - 1, at least 1)
  int32_t slot_stride;      // integer path: every slot_stride-th forward product is kept
  int32_t prefetch;         // integer double-double path: the kernel that reads table values and J entries one step ahead
  int32_t n_polys_total;
  int32_t n_chunks;         // single handle: chunks per polynomial's monomials (>= 1)
  int64_t chunk_f_stride;   // doubles between scratch copies of f
  int64_t chunk_J_stride;   // doubles between scratch copies of J
  double *scratch_f;        // chunk partial results 1 .. n_chunks-1
  double *scratch_J;
  unsigned int *counter;    // work counter (zeroed before each launch)
  int *status;              // device status word
};

struct PowerParams {
  const SysDesc *sys;
  const int64_t *prefix;    // batch: [count+1] prefix sums of n_s * P_s over systems with emax > 2
  const double *points;
  double *table;
  int64_t total;            // number of (system, variable, point) entries
  int32_t count;
  int32_t single_P;         // >= 0: single-system handle
  int32_t single_n;
  int32_t single_emax;
};

// Launchers (kernels.cu).  `dd` selects complex double-double, else complex
// double.  They return the cudaError_t of the launch.
cudaError_t launch_powers(bool dd, const PowerParams &p, cudaStream_t s);
cudaError_t launch_main(bool dd, const MainParams &p, int warps_per_block, size_t smem_bytes, int grid,
                        cudaStream_t s);
cudaError_t main_occupancy(bool dd, bool batch, int warps_per_block, size_t smem_bytes, int *blocks_per_sm);
cudaError_t prepare_main(bool dd, size_t smem_bytes);
cudaError_t fp64_peak_probe(cudaStream_t s, double *fma_per_s, double *sm_clock_mhz);

// Adds the chunk partial results into the outputs and renormalises:
// out[i] = out[i] + scratch_1[i] + ... + scratch_{C-1}[i] for the f and J
// arrays of one system (elements of `doubles_per_elem` doubles).
cudaError_t launch_combine(bool dd, double *out_f, double *out_J, const double *scratch_f, const double *scratch_J,
                           int64_t f_doubles, int64_t J_doubles, int chunks, cudaStream_t s);

// Newton step (newton.cu): solve J dx = -f per point, x += dx.
struct NewtonParams {
  int32_t n;        // variables = polynomials
  int64_t P;        // points
  double *J;        // [n][n][P] Jacobian, factored in place
  double *f;        // [n][P] f on entry, dx on return
  double *x;        // [n][P] points, updated in place
  double *norms;    // [P][2] (|f|_inf, |dx|_inf) or nullptr
  double *Jdd, *fdd;  // quad-double handles: double-double copies of the systems when not staged in shared memory
};
cudaError_t launch_newton(bool dd, const NewtonParams &p, cudaStream_t s);
cudaError_t launch_newton_qd(const NewtonParams &p, cudaStream_t s);
bool newton_qd_needs_scratch(int n);

// The paper's three-kernel design (three_kernel.cu), complex double-double.
struct PaperParams {
  int32_t n, N;      // variables, polynomials
  int32_t M, m, k;   // monomials (N m), monomials per polynomial, variables per monomial
  int32_t d;         // largest exponent
  int32_t P;         // points
  const uint32_t *var;    // [M][k] position | exponent << 16
  const double *coeffs;   // [k + 1][M] complex dd: c a_j (portion j), c (portion k)
  double *cf;             // [P][M] common factors (K1 -> K2)
  double *mons;           // [P][m][N (n + 1)] terms (K2 -> K3)
  const double *points;   // [n][P]
  double *out_f;          // [N][P]
  double *out_J;          // [N][n][P]
};
cudaError_t launch_paper(const PaperParams &p, cudaStream_t s);
cudaError_t prepare_paper(size_t smem_k1, size_t smem_k2);

// Integer-pipe evaluation (kernels_wide.cu): 128-bit block floating point
// products, double-double sums.  Table entries and coefficients are 48 bytes.
constexpr int kWideBytes = 48;
constexpr int kWideSlotBytes = 5 * 4;  // per lane and prefix-product slot
cudaError_t convert_coef_wide(const double *coef_dd, uint32_t *coef_wide, int64_t M, cudaStream_t s);
cudaError_t launch_powers_wide(const PowerParams &p, cudaStream_t s);
cudaError_t prepare_main_wide(size_t smem_bytes);
cudaError_t main_wide_occupancy(bool prefetch, int warps_per_block, size_t smem_bytes, int *blocks_per_sm);
cudaError_t launch_main_wide(const MainParams &p, int warps_per_block, size_t smem_bytes, int grid, cudaStream_t s);

// Quad-double evaluation on the integer pipes (kernels_qd.cu): 256-bit block
// floating point products, 224-bit integer accumulators written in place into
// the outputs, rounded to quad-double by launch_finalize_qd.  Table entries
// and coefficients are 80 bytes.
constexpr int kQdBytes = 80;
constexpr int kQdSlotBytes = 9 * 4;  // per lane and prefix-product slot
cudaError_t convert_coef_qd(const double *coef_qd, uint32_t *coef_blk, int64_t M, cudaStream_t s);
cudaError_t launch_powers_qd(const PowerParams &p, cudaStream_t s);
cudaError_t prepare_main_qd(size_t smem_bytes);
cudaError_t main_qd_occupancy(int warps_per_block, size_t smem_bytes, int *blocks_per_sm);
cudaError_t launch_main_qd(const MainParams &p, int warps_per_block, size_t smem_bytes, int grid, cudaStream_t s);
// Sums the accumulators of `chunks` copies (the outputs, then scratch copies
// 1 .. chunks-1 of the same layout) and rounds them to quad-double in the
// outputs.  Components are 32-byte halves of a complex entry.
cudaError_t launch_finalize_qd(double *out_f, double *out_J, const double *scratch_f, const double *scratch_J,
                               int64_t f_components, int64_t J_components, int chunks, cudaStream_t s);

// Path tracker (track.cu).  Phases of a path and its status (the status
// values are the PE_PATH_* codes of the C ABI).
constexpr int32_t kPhaseCorrect = 0, kPhasePredict = 1, kPhaseEnd = 2;
constexpr int32_t kPathRunning = 0, kPathSuccess = 1, kPathFailed = 2, kPathDiverged = 3, kPathEndNotConverged = 4;

struct TrackState {
  double t;       // last accepted value of the continuation parameter
  double t1;      // value the corrector works at
  double h;       // step size
  double dprev;   // previous corrector step size (contraction check)
  int32_t phase, iter, succ, status;
};

struct TrackParams {
  int32_t n;          // variables = polynomials
  int64_t P;          // paths
  double *J, *f;      // J_F [n][n][P] and F [n][P] at x (evaluator outputs), overwritten
  double *x;          // [n][P] current points
  double *xs;         // [n][P] last accepted point of each path
  double *JL, *bL;    // [n][n][P], [n][P] complex doubles: mixed-precision systems of warp solves in global memory
  TrackState *st;     // [P]
  const int32_t *deg; // [n] degrees of the start system x_i^(d_i) - 1
  double gre, gim;    // gamma
  double h_min, h_max, corr_tol, end_tol, x_big;
  int32_t max_corr, max_end, succ_grow;
  int32_t mixed;      // double-double paths: linear systems solved in double
  unsigned int *active;  // incremented once per path still running after a step
};
cudaError_t launch_track_init(bool dd, const TrackParams &p, double h_init, cudaStream_t s);
cudaError_t launch_track_step(bool dd, const TrackParams &p, cudaStream_t s);
cudaError_t launch_track_finish(const TrackState *st, int64_t P, double *t, int32_t *status, cudaStream_t s);
cudaError_t launch_start_points(bool dd, int32_t n, const int32_t *deg, int64_t first, int64_t P, double *x,
                                cudaStream_t s);
cudaError_t launch_narrow_points(const double *dd, double *c64, int64_t count, cudaStream_t s);
cudaError_t launch_widen_points(const double *c64, double *dd, int64_t count, cudaStream_t s);
cudaError_t launch_move_paths(const double *src, int64_t P_src, double *dst, int64_t P_dst, const int64_t *idx,
                              int64_t m, int32_t n, int words, bool scatter, cudaStream_t s);
cudaError_t launch_scatter_status(const int32_t *src, int32_t *dst, const int64_t *idx, int64_t m, cudaStream_t s);

}  // namespace pe
