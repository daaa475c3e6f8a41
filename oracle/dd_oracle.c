/*
 * Plain CPU double-double evaluator of a sparse polynomial system and its
 * Jacobian -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg load
 * this library.  It shares no code with the CUDA path.
 *
 * It follows the plain definitions of Section 2, Eq. (1) of Verschelde &
 * Yoffe, term by term:
 *     f_p(x)        = sum_t c_t prod_j x_{i_j}^{a_j}
 *     df_p/dx_i(x)  = sum_{t : i in t} c_t a_i x_i^{a_i-1} prod_{j : i_j != i} x_{i_j}^{a_j}
 * Every term is its own product of k powers (no common factor, no
 * Speelpenning prefix products), summed in monomial order.
 *
 * Arithmetic is complex double-double (the precision the paper targets,
 * Sections 1 and 3.2).  The real double-double operations are the textbook
 * error-free transformations:
 *   - TwoSum (Knuth): s = RN(a+b) and the exact error, any magnitudes.
 *   - FastTwoSum (Dekker): same when |a| >= |b|.
 *   - TwoProd with a fused multiply-add: p = RN(ab), e = ab - p exactly.
 *   - Addition of two double-doubles with both error terms propagated
 *     ("accurate" double-word addition, Joldes, Muller & Popescu 2017).
 *   - Product of two double-doubles with the cross terms added by FMA
 *     (double-word times double-word, same paper).
 * The complex product uses the schoolbook form (ac - bd) + i(ad + bc).
 *
 * Must be compiled with -ffp-contract=off so that the compiler fuses no
 * multiply-add the algorithms do not ask for.
 *
 * Layouts (all float64, complex double-double = 4 doubles re_hi, re_lo,
 * im_hi, im_lo):
 *   coef   [M][4]
 *   points [n][P][4]           (variable-major, point-minor)
 *   out_f  [N][P][4]
 *   out_J  [N][n][P][4]
 * Only the points in [q0, q1) are evaluated; other output entries are left
 * untouched.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct { double hi, lo; } dd;
typedef struct { dd re, im; } cdd;

static inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double err = (a - (s - bb)) + (b - bb);
  dd r = {s, err};
  return r;
}

static inline dd fast_two_sum(double a, double b) {
  double s = a + b;
  double err = b - (s - a);
  dd r = {s, err};
  return r;
}

static inline dd two_prod(double a, double b) {
  double p = a * b;
  double e = fma(a, b, -p);
  dd r = {p, e};
  return r;
}

static inline dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  dd t = two_sum(x.lo, y.lo);
  double c = s.lo + t.hi;
  dd v = fast_two_sum(s.hi, c);
  double w = t.lo + v.lo;
  return fast_two_sum(v.hi, w);
}

static inline dd dd_neg(dd x) {
  dd r = {-x.hi, -x.lo};
  return r;
}

static inline dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  double t = x.lo * y.lo;
  t = fma(x.hi, y.lo, t);
  t = fma(x.lo, y.hi, t);
  double c = p.lo + t;
  return fast_two_sum(p.hi, c);
}

static inline dd dd_mul_int(dd x, double k) {
  dd p = two_prod(x.hi, k);
  double c = fma(x.lo, k, p.lo);
  return fast_two_sum(p.hi, c);
}

static inline cdd cdd_mul(cdd x, cdd y) {
  cdd z;
  z.re = dd_add(dd_mul(x.re, y.re), dd_neg(dd_mul(x.im, y.im)));
  z.im = dd_add(dd_mul(x.re, y.im), dd_mul(x.im, y.re));
  return z;
}

static inline cdd cdd_add(cdd x, cdd y) {
  cdd z;
  z.re = dd_add(x.re, y.re);
  z.im = dd_add(x.im, y.im);
  return z;
}

static inline cdd cdd_scale(cdd x, double k) {
  cdd z;
  z.re = dd_mul_int(x.re, k);
  z.im = dd_mul_int(x.im, k);
  return z;
}

static inline cdd cdd_load(const double *p) {
  cdd z = {{p[0], p[1]}, {p[2], p[3]}};
  return z;
}

static inline void cdd_store(double *p, cdd z) {
  p[0] = z.re.hi;
  p[1] = z.re.lo;
  p[2] = z.im.hi;
  p[3] = z.im.lo;
}

static const cdd CDD_ONE = {{1.0, 0.0}, {0.0, 0.0}};
static const cdd CDD_ZERO = {{0.0, 0.0}, {0.0, 0.0}};

/* Evaluate points q0..q1-1.  Returns 0, or -1 on a bad argument / no memory. */
int dd_oracle_eval(int32_t n, int32_t N, const int64_t *poly_ptr, const int64_t *mono_ptr, const int32_t *pos,
                   const int32_t *exps, const double *coef, const double *points, int64_t P, int64_t q0, int64_t q1,
                   double *out_f, double *out_J, int32_t threads) {
  if (n <= 0 || N < 0 || P < 0 || q0 < 0 || q1 > P || q0 > q1) return -1;
  int32_t emax = 1;
  int64_t nnz = mono_ptr[poly_ptr[N]];
  for (int64_t i = 0; i < nnz; i++) {
    if (exps[i] < 1 || pos[i] < 0 || pos[i] >= n) return -1;
    if (exps[i] > emax) emax = exps[i];
  }
  int status = 0;
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel
#endif
  {
    /* powers x_v^e, e = 0..emax, for one point */
    cdd *pw = (cdd *)malloc(sizeof(cdd) * (size_t)n * (size_t)(emax + 1));
    if (!pw) {
#ifdef _OPENMP
#pragma omp atomic write
#endif
      status = -1;
    } else {
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 1)
#endif
      for (int64_t q = q0; q < q1; q++) {
        for (int32_t v = 0; v < n; v++) {
          cdd xv = cdd_load(points + ((size_t)v * P + q) * 4);
          pw[(size_t)v * (emax + 1)] = CDD_ONE;
          for (int32_t e = 1; e <= emax; e++)
            pw[(size_t)v * (emax + 1) + e] = cdd_mul(pw[(size_t)v * (emax + 1) + e - 1], xv);
        }
        for (int32_t p = 0; p < N; p++) {
          cdd fp = CDD_ZERO;
          for (int32_t i = 0; i < n; i++) cdd_store(out_J + (((size_t)p * n + i) * P + q) * 4, CDD_ZERO);
          for (int64_t t = poly_ptr[p]; t < poly_ptr[p + 1]; t++) {
            int64_t b = mono_ptr[t], e = mono_ptr[t + 1];
            cdd c = cdd_load(coef + (size_t)t * 4);
            /* value term c * prod x^a */
            cdd term = c;
            for (int64_t j = b; j < e; j++) term = cdd_mul(term, pw[(size_t)pos[j] * (emax + 1) + exps[j]]);
            fp = cdd_add(fp, term);
            /* derivative terms c * a_i * x_i^(a_i-1) * prod_{j != i} x^a */
            for (int64_t i = b; i < e; i++) {
              cdd d = cdd_scale(c, (double)exps[i]);
              for (int64_t j = b; j < e; j++) {
                int32_t a = (j == i) ? exps[j] - 1 : exps[j];
                d = cdd_mul(d, pw[(size_t)pos[j] * (emax + 1) + a]);
              }
              double *dst = out_J + (((size_t)p * n + pos[i]) * P + q) * 4;
              cdd_store(dst, cdd_add(cdd_load(dst), d));
            }
          }
          cdd_store(out_f + ((size_t)p * P + q) * 4, fp);
        }
      }
      free(pw);
    }
  }
  return status;
}

/* Number of OpenMP threads a parallel region would use (1 without OpenMP). */
int dd_oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
