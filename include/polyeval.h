/*
 * polyeval -- evaluation of a sparse polynomial system and its full Jacobian
 * at many points on one GB300 GPU (sm_103a), in complex double-double,
 * complex quad-double or complex double precision.
 *
 * The method is the one of Verschelde & Yoffe, "Evaluating polynomials in
 * several variables and their derivatives on a GPU computing processor":
 *   - Section 2, Eq. (1): a polynomial is a tuple (C, A) of nonzero complex
 *     coefficients and exponent vectors; a system is a tuple of polynomials.
 *   - Section 2 (three stages) and Section 3.1: each monomial x^a is the
 *     common factor prod x_{i_j}^{a_j - 1} (read from a table of powers)
 *     times the Speelpenning product x_{i_1} ... x_{i_k}.
 *   - Section 3.2: the gradient of the Speelpenning product from forward
 *     prefix products and one backward running product.
 *   - Section 3.3: coefficient products and the sums into f and J.
 *
 * Conventions for every entry point:
 *   - Return value: PE_OK (0) or a negative PE_E* code; nothing aborts and no
 *     C++ exception crosses this interface.  polyeval_strerror() names codes.
 *   - "device" pointers are CUDA global-memory addresses on the current
 *     device; "host" pointers are ordinary CPU memory.  Device arrays of
 *     points, coefficients and outputs must be 16-byte aligned (cudaMalloc
 *     and torch allocations are); a misaligned one is PE_EINVAL.
 *   - Streams are passed as `void *` holding a cudaStream_t (NULL = legacy
 *     default stream).  Every eval call is asynchronous on that stream.
 *   - All sizes are element counts unless stated.
 *   - A handle owns device scratch (power table, monomial-chunk partial sums,
 *     solver and tracker buffers) that every call on it reuses: calls on one
 *     handle must not overlap, neither from several host threads nor on
 *     several streams without ordering between them.  Different handles are
 *     independent.
 *
 * Data layouts (structure of arrays, point index fastest):
 *   - A complex double-double (pe_cdd) is 4 doubles: re_hi, re_lo, im_hi,
 *     im_lo; the value is (re_hi + re_lo) + i (im_hi + im_lo).  A complex
 *     quad-double (pe_cqd) is 8 doubles: re[0..3], im[0..3]; the value is
 *     (re[0] + re[1] + re[2] + re[3]) + i (im[0] + ... + im[3]).  A complex
 *     double (pe_c64) is 2 doubles: re, im.
 *   - points: [n_vars][P] entries (entry (v, q) at index v * P + q).
 *   - out_f : [n_polys][P]          (f_p at point q at index p * P + q).
 *   - out_J : [n_polys][n_vars][P]  (d f_p / d x_i at point q at index
 *             (p * n_vars + i) * P + q).
 *   Entries of J for a variable that does not occur in polynomial p are
 *   written as exact zeros.
 *
 * Accuracy (normwise, against the exact result, relative to the same sum
 * over absolute values: sum |c| |x^a| for f, sum |c| a_i |x^(a - e_i)| for
 * J): <= 1e-28 for PE_DD and PE_DD_INT, <= 1e-60 for PE_QD_INT and <= 1e-13
 * for PE_F64 on the workloads this library is tested on; see the tests for
 * the exact cases.
 */
#ifndef POLYEVAL_H
#define POLYEVAL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Exported symbols of the shared library (everything else is hidden). */
#if defined(__GNUC__)
#define PE_API __attribute__((visibility("default")))
#else
#define PE_API
#endif

/* ---- status codes ------------------------------------------------------ */
#define PE_OK 0
#define PE_EINVAL (-1)  /* bad argument or malformed system                  */
#define PE_ENOMEM (-2)  /* host or device allocation failed                  */
#define PE_ECUDA (-3)   /* a CUDA runtime call failed (see cudaGetLastError)  */
#define PE_ERANGE (-4)  /* a size above the limits of this build             */
#define PE_EDEVICE (-5) /* a kernel reported an inconsistency (status word)  */

/* ---- precisions -------------------------------------------------------- */
#define PE_DD 0  /* complex double-double (pe_cdd in and out)  */
#define PE_F64 1 /* complex double        (pe_c64 in and out)  */
/* Complex double-double in and out (pe_cdd), products computed in complex
 * block floating point with 128-bit integer mantissas on the integer pipes
 * (error about 2^-120 per product relative to the operands' magnitudes),
 * sums in double-double.  Same method and layouts as PE_DD; more accurate
 * and, on GB300 where FP64 issues about 36x slower than integer multiply-add,
 * faster. */
#define PE_DD_INT 2
/* Complex quad-double in and out (pe_cqd), the precision of the QD library
 * the paper's CPU code uses (Section 1).  Products in complex block floating
 * point with 256-bit integer mantissas (error about 2^-246 per product
 * relative to the operands' magnitudes); every sum in a 224-bit integer
 * accumulator per output component, kept in place in the output arrays and
 * rounded to quad-double (each part the nearest double to what the parts
 * before it leave) by a final pass.  No FP64 arithmetic.  Coefficients come
 * from pe_system.coef_qd, or from coef (lower parts zero) when coef_qd is
 * NULL.  polyeval_newton and PE_PAPER_KERNELS reject this precision. */
#define PE_QD_INT 3

/* ---- flags for polyeval_create / polyeval_create_many / polyeval_validate */
#define PE_ALLOW_ZERO_COEF 1u /* accept c = 0 (Eq. 1 asks c != 0); for tests */
/* Evaluate with the paper's own three-kernel design (Sections 3.1-3.3: common
 * factors to global memory, Speelpenning products and coefficient products
 * scattered into a zero-padded term array, one thread per output summing m
 * terms) instead of the fused kernel, for comparison.  PE_DD only; regular
 * systems only (every polynomial the same number m of monomials, every
 * monomial the same number k >= 3 of variables) and max_points <= 65535,
 * else PE_EINVAL.  The term array takes (n^2 + n) m complex double-doubles
 * per point of max_points. */
#define PE_PAPER_KERNELS 2u

/* ---- limits ------------------------------------------------------------ */
#define PE_MAX_VARS 65535 /* n_vars                                        */
#define PE_MAX_EXP 256    /* largest exponent a (the paper stores a-1 in a byte) */

typedef struct {
  double re_hi, re_lo, im_hi, im_lo;
} pe_cdd;

typedef struct {
  double re, im;
} pe_c64;

typedef struct {
  double re[4], im[4];
} pe_cqd;

/*
 * A polynomial system in compressed rows (Section 2, Eq. 1; the monomial
 * order of Section 3.3: the monomials of polynomial 0, then of polynomial 1,
 * ...).  All arrays are host memory owned by the caller.
 *   n_vars     number of variables n >= 1
 *   n_polys    number of polynomials N >= 0
 *   poly_ptr   [N + 1]   monomials of polynomial p are poly_ptr[p] ..
 *                        poly_ptr[p+1]-1; poly_ptr[0] = 0, nondecreasing
 *   mono_ptr   [M + 1]   (M = poly_ptr[N]) variables of monomial t are
 *                        entries mono_ptr[t] .. mono_ptr[t+1]-1 of pos/exp;
 *                        mono_ptr[0] = 0, nondecreasing.  k = 0 (a constant
 *                        term) and k = 1 are allowed.
 *   pos        variable index 0 <= pos < n, strictly increasing inside a
 *              monomial (i_1 < i_2 < ... < i_k)
 *   exp        exponent 1 <= a <= PE_MAX_EXP
 *   coef       [M] coefficients, nonzero and finite.  For PE_F64 only the
 *              high words are read.  May be NULL when coef_qd is given and the
 *              precision is PE_QD_INT.
 *   coef_qd    [M] quad-double coefficients, nonzero and finite, or NULL.
 *              Read only by PE_QD_INT (which then ignores coef).
 */
typedef struct {
  int32_t n_vars;
  int32_t n_polys;
  const int64_t *poly_ptr;
  const int64_t *mono_ptr;
  const int32_t *pos;
  const int32_t *exp;
  const pe_cdd *coef;
  const pe_cqd *coef_qd;
} pe_system;

typedef struct polyeval polyeval_t;

/*
 * Check a system on the host only (no CUDA call).  The coefficients checked
 * are coef, or coef_qd when coef is NULL.  Returns PE_OK, PE_EINVAL
 * (null pointer, n_vars < 1, n_polys < 0, offsets not starting at 0 or
 * decreasing, pos out of range / not strictly increasing, exponent < 1,
 * zero or non-finite coefficient without PE_ALLOW_ZERO_COEF) or PE_ERANGE
 * (n_vars > PE_MAX_VARS, exponent > PE_MAX_EXP, more than 2^31-1 monomials or
 * variable entries).
 */
PE_API int polyeval_validate(const pe_system *sys, uint32_t flags);

/*
 * Compile one system for evaluation (Section 2 format -> device metadata).
 *   sys         host system, copied; the caller may free it on return
 *   precision   PE_DD, PE_F64, PE_DD_INT or PE_QD_INT
 *   flags       PE_ALLOW_ZERO_COEF or 0
 *   max_points  largest P any later polyeval_eval call will pass (>= 1);
 *               sizes the table of powers (Section 3.1) kept on the device
 *   out         receives the handle; *out is NULL on failure
 * The handle owns all device memory it allocates (metadata, power table,
 * work counter, status word); polyeval_destroy frees it.  Errors: those of
 * polyeval_validate, PE_EINVAL for a bad precision/max_points/out,
 * PE_ENOMEM, PE_ECUDA, PE_ERANGE when a monomial has more variables than the
 * shared-memory prefix store of one warp can hold.
 */
PE_API int polyeval_create(const pe_system *sys, int precision, uint32_t flags, int64_t max_points, polyeval_t **out);

/*
 * Evaluate f and J at P points (Sections 3.1-3.3).
 *   points  device, [n_vars][P] pe_cdd (PE_DD, PE_DD_INT), pe_cqd (PE_QD_INT)
 *           or pe_c64 (PE_F64)
 *   P       number of points, 0 <= P <= max_points (0 returns PE_OK at once)
 *   out_f   device, [n_polys][P] of the same element type
 *   out_J   device, [n_polys][n_vars][P] of the same element type
 *   stream  cudaStream_t the work is queued on
 * Allocates nothing, synchronises nothing, and only queues kernels and one
 * 4-byte cudaMemsetAsync, so a call can be captured in a CUDA graph.  When
 * the call has few (polynomial, tile of 16 points) work items, each
 * polynomial's monomials are split into up to 8 chunks whose partial sums go
 * to handle-owned scratch (at most 256 MiB, sized at create) and are added
 * by a final kernel (for PE_QD_INT the final kernel always runs: it rounds
 * the integer sums in the outputs to quad-double, so the outputs hold
 * intermediate sums until it completes).  Calls on one handle must not overlap on the GPU (they
 * share the power table, the scratch and the work counter).  Errors: PE_EINVAL (null handle/pointer with P > 0),
 * PE_ERANGE (P > max_points), PE_ECUDA (launch failure).
 */
PE_API int polyeval_eval(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream);

/*
 * Choose the launch of polyeval_eval for P points by timing the candidates on
 * the caller's data: the number of chunks the monomials of each polynomial
 * are split into (1, 2, 4, 8, as the handle's scratch allows), the launch
 * shape (1: one single-warp block per work item, all resident at once; 2: a
 * persistent grid taking items from the work counter) and, for PE_DD and
 * PE_F64 calls with fewer than 64 points, the threads per monomial: groups
 * G = 1, 2, 4, 8, 16 of a warp work on G monomials at once, each group of
 * 32 / G lanes on 16 / G points.  Runs each candidate four times on `stream`
 * (one warm-up, three timed with CUDA events), synchronises, keeps the
 * fastest in the handle for later calls with the same P, and returns it in
 * *chunks, *shape and *groups (any may be NULL).  The outputs hold a valid
 * evaluation on return.  Not for use during stream capture.  Errors: those of
 * polyeval_eval.
 *
 * Batch handles (polyeval_create_many): pass P = 0 and the batch buffers of
 * polyeval_eval_many.  The candidates are the monomial chunks of every
 * (polynomial, tile) item (1, 2, 4, 8, as the handle's chunk scratch allows:
 * at create a batch handle allocates min(7 copies of all its f and J,
 * 256 MiB) when that holds at least one copy), the launch shape, and for
 * PE_DD and PE_F64 the monomial groups of a system's partial last tile
 * (*groups = 16: a tile of r < 16 points takes the largest G with G r <= 16
 * groups of 32 / G lanes; *groups = 1: one group, lane pairs past r idle).
 * The choice is kept for polyeval_eval_many.  Before a change of the
 * partial-tile groups the call waits for all work on the device and rewrites
 * the handle's item table.  Errors as for single handles; PE_EINVAL for
 * P != 0.
 */
PE_API int polyeval_autotune(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream,
                             int *chunks, int *shape, int *groups);

/*
 * Set the launch polyeval_eval uses for calls with exactly P points (what
 * polyeval_autotune would store): chunks 1..8 monomial chunks per polynomial
 * (capped by the handle's scratch at run time), shape 1 (one single-warp
 * block per work item) or 2 (persistent grid), and groups 1, 2, 4, 8 or 16
 * monomial groups per warp (PE_DD and PE_F64; ignored by the integer-pipe
 * precisions).  0 for any leaves that choice to the built-in heuristic (for
 * groups: the largest G with G P <= 16); all 0 removes the entry.
 * Batch handles: P = 0; chunks and shape as above for polyeval_eval_many,
 * groups the most monomial groups of a partial last tile (0 or 16: as many as
 * fill the warp, the built-in choice); the call waits for all work on the
 * device when it rewrites the item table.  Errors: PE_EINVAL; PE_ECUDA.
 */
PE_API int polyeval_set_launch(polyeval_t *h, int64_t P, int chunks, int shape, int groups);

/*
 * One Newton step x <- x + dx, J(x) dx = -f(x), at P points of a square
 * system (n_polys == n_vars).  Evaluating f and J is the expensive part of
 * Newton's method, the corrector of a path tracker (Section 1); this entry
 * point adds the linear solve so that a caller can correct a batch of
 * points in one call.
 *   points  device [n][P], updated in place (points whose Jacobian has an
 *           exact zero pivot column are left unchanged)
 *   out_f   device [n][P]: on return dx (not f)
 *   out_J   device [n][n][P]: on return the LU factors (unit lower triangle
 *           below the diagonal, after the row exchanges of partial pivoting)
 *   norms   device [P][2] doubles or NULL: max_i |f_i(x)| before the step and
 *           max_i |dx_i| (NaN for a singular point)
 *   stream  as polyeval_eval
 * The solve is LU with partial pivoting per point (pivot of largest modulus)
 * in the handle's precision (double-double for PE_DD and PE_DD_INT, double
 * for PE_F64), 4 to 32 lanes of a warp per point.  PE_QD_INT handles
 * evaluate f and J in quad-double and solve for dx in double-double from
 * the leading two parts of each component (mixed precision, as iterative
 * refinement: each step gains about 104 bits less log2 cond(J) until x
 * reaches quad-double accuracy); x + dx is summed exactly and rounded to
 * quad-double.  There out_f holds dx with parts 2, 3 zero and out_J the
 * double-double factors in parts 0, 1 (parts 2, 3 zero).  Allocates nothing,
 * except on a PE_QD_INT handle with n > 22, whose first call allocates
 * 32 n (n + 1) max_points bytes of double-double scratch for the handle.
 * Errors: those of polyeval_eval; PE_EINVAL for a batch handle or a
 * non-square system; PE_ENOMEM when that scratch cannot be allocated.
 */
PE_API int polyeval_newton(polyeval_t *h, void *points, int64_t P, void *out_f, void *out_J, double *norms,
                           void *stream);

/*
 * polyeval_eval with HOST buffers: copies points to the device, evaluates,
 * and copies f and J back, then synchronises.  When the outputs of the call
 * exceed 512 MiB the points are split into C chunks (one per 256 MiB of
 * outputs, at most 8, each of at least 1024 points): chunk c is evaluated on
 * `stream` while the outputs of chunk c - 1 are copied to the host on a
 * stream of the handle, so the copies hide behind the evaluation; each
 * chunk's columns of the [.][P] host arrays are moved by one pitched copy.
 * The results are those of polyeval_eval on the chunks' point counts.
 * Host buffers should be pinned for full copy speed and for the overlap.
 * Device staging buffers (two chunks' worth when split) are allocated on the
 * first call (and grown when P grows) and kept by the handle.  Errors: as
 * polyeval_eval, plus PE_ENOMEM.
 */
PE_API int polyeval_eval_host(polyeval_t *h, const void *points, int64_t P, void *out_f, void *out_J, void *stream);

/*
 * Compile a batch of systems of uneven shape, to be evaluated in one
 * persistent launch (each system at its own set of points).
 *   systems            [count] host systems (copied)
 *   count              >= 1
 *   points_per_system  [count] P_s >= 0 points for each system
 * The device buffers of a batch are single arrays with every system's block
 * at a fixed offset; polyeval_many_layout() returns the offsets.  Work items
 * (polynomial, tile of points) are ordered by decreasing cost.  Errors: as
 * polyeval_create.
 */
PE_API int polyeval_create_many(const pe_system *systems, int32_t count, int precision, uint32_t flags,
                         const int64_t *points_per_system, polyeval_t **out);

/*
 * Offsets of system s inside the batch buffers, in elements (pe_cdd or
 * pe_c64): its points start at points + *pt_off and are laid out
 * [n_s][P_s]; its f at out_f + *f_off ([N_s][P_s]); its J at out_J + *J_off
 * ([N_s][n_s][P_s]).  Any of the output pointers may be NULL.  With s = count
 * the offsets are the total sizes (elements are pe_cqd for PE_QD_INT).  Errors: PE_EINVAL (not a batch handle,
 * s out of range).
 */
PE_API int polyeval_many_layout(const polyeval_t *h, int32_t s, int64_t *pt_off, int64_t *f_off, int64_t *J_off);

/*
 * Evaluate every system of a batch handle.  points, out_f and out_J are the
 * device batch buffers laid out as polyeval_many_layout() describes.  Same
 * asynchrony and graph-capture properties as polyeval_eval.
 */
PE_API int polyeval_eval_many(polyeval_t *h, const void *points, void *out_f, void *out_J, void *stream);

/*
 * Work counts of the handle, per evaluation point and summed over the
 * handle's systems (for a batch: over all points of all systems, i.e. one
 * whole polyeval_eval_many):
 *   fp64_ops    double-precision instructions (add, mul, fma) the method
 *               executes, counted from the compiled system (for PE_DD_INT:
 *               those of its double-double sums; 0 for PE_QD_INT, which
 *               has none)
 *   fp64_flops  the same with an fma counted as 2 flops
 * Either pointer may be NULL.
 */
PE_API int polyeval_cost(const polyeval_t *h, double *fp64_ops, double *fp64_flops);

/*
 * Timing of the main (monomial) kernel, for measurement.  With enable != 0,
 * each following eval call records a pair of CUDA events on its stream
 * around the main kernel (at most 256 pairs are kept).  polyeval_timing_read
 * waits for the recorded events, returns the summed kernel time in
 * milliseconds, the number of timed launches and the number of kernels the
 * eval calls queued (power table, main kernel, combine passes), and starts a
 * new count.  Returns PE_ERANGE if launches beyond the 256 kept pairs went
 * untimed.  Any output pointer may be NULL.
 */
PE_API int polyeval_timing(polyeval_t *h, int enable);
PE_API int polyeval_timing_read(polyeval_t *h, double *total_ms, int64_t *launches, int64_t *kernels);

/*
 * Read and clear the device status word (synchronises the device).
 * Returns PE_OK, or PE_EDEVICE if a kernel found an inconsistent index.
 */
PE_API int polyeval_status(polyeval_t *h);

/*
 * Evaluation for callers that cannot allocate device memory.  (This entry
 * point has no counterpart in the paper; it is a deployment variant of
 * polyeval_eval.)
 *
 * A caller whose device memory belongs to another allocator (a framework's
 * caching allocator, a pre-reserved arena, a fixed start-up budget) cannot
 * let this library call cudaMalloc, and so cannot use polyeval_create.  This
 * entry point allocates nothing: the caller passes the system, the points
 * and the outputs in its own device memory, and the only scratch -- the
 * table of powers x^2 .. x^(d-1) of every variable at every point -- lives
 * in a static 16 MiB device array that every GPU loading the library holds
 * until the process exits.
 *
 *   dev_sys   host struct in the pe_system format whose pointer fields
 *             (poly_ptr, mono_ptr, pos, exp, coef) are DEVICE pointers; the
 *             arrays must satisfy what polyeval_validate checks (they are not
 *             read on the host)
 *   max_k     an upper bound on the variables of any monomial (<= 256)
 *   max_exp   an upper bound on any exponent (<= PE_MAX_EXP)
 *   points, P, out_f, out_J, stream   as polyeval_eval, complex
 *             double-double (pe_cdd) only
 * Limits: (max_exp - 2) * n_vars * P complex double-doubles must fit in the
 * 16 MiB array (524288 of them), else PE_ERANGE; PE_EINVAL for null pointers
 * or negative sizes.  A monomial breaking max_k, max_exp or 0 <= pos < n is
 * skipped and f of its polynomial is written as NaN.
 * Each one-warp block takes (max_k - 1) * 512 bytes of shared memory (one
 * forward-product slot per variable and lane), so the bound sets how many
 * warps share an SM: pass the smallest max_k that holds (max_k = 256 takes
 * about 130 KB, one warp per SM; 32 takes 16 KB).
 * The first call on a device looks up the array's device address (and sets
 * the kernel's shared-memory limit) with that device current and keeps both
 * for the life of the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) after it is not supported: the
 * kept address and limit belong to the context the reset destroys.  Every call uses the same array:
 * each call writes all the table entries it reads before reading them, so
 * nothing has to start at zero, but calls that overlap on the GPU (other
 * streams or host threads) race on it.
 */
PE_API int polyeval_eval_noalloc(const pe_system *dev_sys, int32_t max_k, int32_t max_exp, const void *points,
                                 int64_t P, void *out_f, void *out_J, void *stream);

/* ---- path tracking ------------------------------------------------------
 *
 * Solving F(x) = 0 (a square system, n_polys == n_vars) by homotopy
 * continuation, the application the paper's evaluation serves (Section 1:
 * evaluation inside Newton's method, the corrector of a path tracker; only a
 * few paths need double-double).  The homotopy is
 *     H(x, t) = gamma (1 - t) G(x) + t F(x),   G_i(x) = x_i^(d_i) - 1,
 * with d_i the total degree of polynomial i and gamma a complex constant
 * (for generic gamma every path is regular on [0, 1)).  The start solutions
 * are the prod d_i points whose coordinates are roots of unity.  Every path
 * is one point of the evaluator's batch; one iteration evaluates F and J_F
 * at all points (polyeval_eval) and then advances each path by one step of
 * its own state machine (4 to 32 lanes of a warp per path, as n and the
 * batch size call for): Newton corrector at t1
 * (accepted when max|dx| <= corr_tol max(1, max|x|) within max_corr steps
 * that keep shrinking, else rejected: back to the last accepted point, step
 * size halved, failed below h_min), Euler predictor along the tangent
 * (H_x v = -H_t, t1 = min(t + h, 1)), step size doubled after succ_grow
 * accepted steps in a row (at most h_max), and at t = 1 Newton's method on
 * F until max|dx| <= end_tol max(1, max|x|) (at most max_end steps).
 * With `mixed` set, a double-double tracker keeps the homotopy, residuals and
 * points in double-double but solves its linear systems in double from the
 * leading parts of H_x (each Newton step is then a step of iterative
 * refinement), which takes about a tenth of the FP64 work of a double-double
 * solve (the handle keeps an n x n x P double scratch for it).
 */
typedef struct {
  double gamma_re, gamma_im; /* gamma (nonzero)                                   */
  double h_init, h_min, h_max; /* step sizes in t                                   */
  double corr_tol, end_tol;  /* relative step tolerances (see above)              */
  double x_big;              /* max|x| above which a path counts as diverging     */
  int32_t max_corr, max_end, succ_grow;
  int32_t mixed;             /* double-double handles: solve in double (see above) */
  int64_t max_iters;         /* iterations (evaluations) of the whole batch, at most */
} pe_track_params;

/* Status of a path after polyeval_track / polyeval_track_adaptive. */
#define PE_PATH_RUNNING 0       /* max_iters reached first                         */
#define PE_PATH_SUCCESS 1       /* reached t = 1 and converged there               */
#define PE_PATH_FAILED 2        /* step size fell below h_min                      */
#define PE_PATH_DIVERGED 3      /* max|x| exceeded x_big, or x or dx not finite    */
#define PE_PATH_END_NOT_CONVERGED 4 /* at t = 1 Newton did not reach end_tol (singular or ill-conditioned end point) */

/* Default tracking parameters for a precision (PE_DD, PE_DD_INT or PE_F64):
 * gamma = exp(i), h_init 0.02, h_min 1e-14 (double-double) or 1e-10, h_max 0.1,
 * corr_tol 1e-6, end_tol 1e-26 (double-double) or 1e-13, x_big 1e8,
 * max_corr 3, max_end 8, succ_grow 3, mixed 1 for double-double,
 * max_iters 100000. */
PE_API int polyeval_track_defaults(int precision, pe_track_params *prm);

/* The Bezout number prod d_i (the number of paths) as a double, and the
 * degrees d_i into degrees[n] (either may be NULL).  Single-system handles. */
PE_API int polyeval_bezout(const polyeval_t *h, double *count, int32_t *degrees);

/*
 * Start solutions of G(x) = 0 for paths first .. first + P - 1 into the
 * device array points [n][P] (pe_cdd or pe_c64 as the handle's precision):
 * path r has coordinates x_i = exp(2 pi i k_i / d_i) with k_i the mixed-radix
 * digits of r (radices d_0, d_1, ...).  Asynchronous on stream.  Errors:
 * PE_EINVAL for a handle that cannot track (batch, PE_QD_INT, paper
 * kernels, not square, a polynomial of degree 0) or bad arguments.
 */
PE_API int polyeval_start_points(polyeval_t *h, int64_t first, int64_t P, void *points, void *stream);

/*
 * Track P paths from the start points in `points` (device [n][P], the
 * handle's precision; on return the end points) from t = 0 to t = 1.
 *   t, status   device [P] arrays (either may be NULL): the last accepted t
 *               and the PE_PATH_* status of each path
 *   iterations  host, or NULL: iterations the batch took
 * Blocks the calling thread: it synchronises `stream` (so that the start
 * points are in place), then runs the iterations on a stream of the
 * handle's own, replaying batches of 8 iterations from a CUDA graph captured
 * on the first call, reads how many paths still run after each batch, and
 * returns when none does (or after max_iters) with all its work complete.
 * Allocates the tracker's scratch and stream on the handle on first use (F,
 * J_F, saved points, path states for P paths).  Not for stream capture.
 * Errors: PE_EINVAL (as polyeval_start_points, bad parameters), PE_ERANGE
 * (P > max_points), PE_ENOMEM, PE_ECUDA.
 */
PE_API int polyeval_track(polyeval_t *h, const pe_track_params *prm, void *points, int64_t P, double *t,
                          int32_t *status, int64_t *iterations, void *stream);

/*
 * Adaptive precision: every path is tracked in double (h_lo, a PE_F64 handle
 * of the system); the end points of the paths that succeed are refined by
 * three Newton steps in double-double (h_hi, a PE_DD or PE_DD_INT handle of
 * the same system), and only the paths that did not succeed are tracked
 * again, from their start points, in double-double (with their linear systems
 * in double-double whatever prm_hi->mixed says: these are the hard paths).
 *   points     device [n][P] pe_cdd: start points in, end points out
 *   status     device [P]: PE_PATH_* of each path (of its final tracking)
 *   escalated  host, or NULL: the number of paths tracked in double-double
 * Blocks like polyeval_track.  Errors: PE_EINVAL (wrong precisions, systems
 * of different shape or degrees, bad parameters), PE_ERANGE, PE_ENOMEM,
 * PE_ECUDA.
 */
PE_API int polyeval_track_adaptive(polyeval_t *h_lo, polyeval_t *h_hi, const pe_track_params *prm_lo,
                                   const pe_track_params *prm_hi, void *points, int64_t P, int32_t *status,
                                   int64_t *escalated, void *stream);

/* Free a handle and its device memory (NULL is accepted). */
PE_API void polyeval_destroy(polyeval_t *h);

/* Static string naming a status code. */
PE_API const char *polyeval_strerror(int code);

/*
 * Measure the double-precision FMA issue rate of the current device: a
 * short (about 2 ms) kernel of independent FMA chains on every SM, timed
 * with CUDA events on `stream` (synchronises the stream).  *fma_per_s
 * receives lane-FMAs per second; *sm_clock_mhz the SM clock implied by the
 * kernel's cycle counter.  Used as the denominator of the FP64 roofline.
 */
PE_API int polyeval_fp64_peak(void *stream, double *fma_per_s, double *sm_clock_mhz);

#ifdef __cplusplus
}
#endif

#endif /* POLYEVAL_H */
