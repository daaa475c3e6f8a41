"""Exact CPU oracle for f(x) and its Jacobian.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module;
only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may use it.

It evaluates the plain definitions of Section 2, Eq. (1) of Verschelde & Yoffe:

    f_p(x)          = sum_{a in A_p} c_a x^a,      x^a = prod_i x_i^{a_i}
    d f_p / d x_i   = sum_{a in A_p, a_i >= 1} c_a a_i x_i^{a_i - 1} prod_{j != i} x_j^{a_j}

term by term, for every point, with no common factors, no Speelpenning
products and no reordering: each term is the product written out.

Every input is a double, a double-double or a quad-double (a sum of two or
four doubles), hence a dyadic rational, so the arithmetic here is exact: a complex number is held as (A + iB) * 2**E with
Python integers A, B, E.  Nothing is rounded until an error is measured.

The normwise error of a computed output z against the exact value z* is
|z - z*| / S, with S the same sum taken over absolute values
(S_f = sum |c| |x^a|; S_J = sum |c| a_i |x^(a - e_i)|).  S is a scale for a
tolerance and is computed in float64.
"""
from __future__ import annotations

import math
from typing import Sequence, Tuple

# ----------------------------------------------------------------------------
# exact complex dyadic numbers: (A, B, E) means (A + iB) * 2**E
# ----------------------------------------------------------------------------

ZERO = (0, 0, 0)
ONE = (1, 0, 0)


def dyadic(x: float) -> Tuple[int, int]:
    """A double as (M, E) with x = M * 2**E exactly."""
    if x == 0.0:
        return 0, 0
    num, den = float(x).as_integer_ratio()  # den is a power of two
    return num, -(den.bit_length() - 1)


def real_dd(hi: float, lo: float) -> Tuple[int, int]:
    """hi + lo exactly, as (M, E)."""
    return real_sum((hi, lo))


def real_sum(parts: Sequence[float]) -> Tuple[int, int]:
    """The exact sum of any doubles, as (M, E)."""
    ds = [dyadic(float(x)) for x in parts]
    e = min(d[1] for d in ds)
    return sum(m << (x - e) for m, x in ds), e


def cx_from_dd(v: Sequence[float]):
    """A complex multi-double exactly: 4 values (re_hi, re_lo, im_hi, im_lo)
    for a double-double, 8 (re0..re3, im0..im3) for a quad-double; each
    component is the exact sum of its parts."""
    w = len(v) // 2
    a, ea = real_sum(v[:w])
    b, eb = real_sum(v[w:2 * w])
    e = min(ea, eb)
    return (a << (ea - e), b << (eb - e), e)


def cx_mul(x, y):
    """(a + ib)(c + id) = (ac - bd) + i(ad + bc); exponents add."""
    a, b, e = x
    c, d, f = y
    return (a * c - b * d, a * d + b * c, e + f)


def cx_add(x, y):
    """Sum after aligning both to the smaller exponent."""
    a, b, e = x
    c, d, f = y
    if e <= f:
        s = f - e
        return (a + (c << s), b + (d << s), e)
    s = e - f
    return ((a << s) + c, (b << s) + d, f)


def cx_scale(x, k: int):
    """Multiply by an integer."""
    return (x[0] * k, x[1] * k, x[2])


def cx_sub(x, y):
    return cx_add(x, (-y[0], -y[1], y[2]))


def cx_equal(x, y) -> bool:
    d = cx_sub(x, y)
    return d[0] == 0 and d[1] == 0


def _int_to_float_scaled(m: int, e: int) -> float:
    """m * 2**e rounded to the nearest double (ties to even).

    CPython's int -> float conversion is correctly rounded; for very long m
    the discarded bits are first folded into a sticky bit so that the single
    rounding still sees them.  Results beyond the double range give inf."""
    if m == 0:
        return 0.0
    bl = abs(m).bit_length()
    if bl > 64:
        sh = bl - 64
        mag = abs(m)
        kept = (mag >> sh) | (1 if mag & ((1 << sh) - 1) else 0)
        m = kept if m > 0 else -kept
        e += sh
    try:
        return math.ldexp(float(m), e)
    except OverflowError:
        return math.copysign(math.inf, m)


def cx_abs(x) -> float:
    a, b, e = x
    return math.hypot(_int_to_float_scaled(a, e), _int_to_float_scaled(b, e))


def cx_to_dd(x) -> Tuple[float, float, float, float]:
    """Round an exact value to a complex double-double (hi = RN(v), lo = RN(v - hi))."""
    out = []
    for m in (x[0], x[1]):
        hi = _int_to_float_scaled(m, x[2])
        mh, eh = dyadic(hi)
        e = min(eh, x[2])
        rest = (m << (x[2] - e)) - (mh << (eh - e))
        lo = _int_to_float_scaled(rest, e)
        out.extend([hi, lo])
    return tuple(out)


def real_to_parts(m: int, e: int, parts: int):
    """m * 2**e as `parts` doubles: each the nearest double to what the parts
    before it leave (a normalised multi-double)."""
    out = []
    for _ in range(parts):
        d = _int_to_float_scaled(m, e)
        out.append(d)
        md, ed = dyadic(d)
        emin = min(ed, e)
        m = (m << (e - emin)) - (md << (ed - emin))
        e = emin
    return out


def cx_to_qd(x) -> Tuple[float, ...]:
    """Round an exact value to a complex quad-double (re0..re3, im0..im3),
    each component a normalised sum of four doubles."""
    return tuple(real_to_parts(x[0], x[2], 4) + real_to_parts(x[1], x[2], 4))


# ----------------------------------------------------------------------------
# evaluation by definition (Section 2, Eq. 1)
# ----------------------------------------------------------------------------

def powers_of(xv, top: int):
    """[x^0, x^1, ..., x^top] by repeated multiplication."""
    out = [ONE]
    for _ in range(top):
        out.append(cx_mul(out[-1], xv))
    return out


class _LazyPowers:
    """Powers [x_v^0 .. x_v^top] of each variable, made on first use."""

    def __init__(self, pts, q, top):
        self.pts, self.q, self.top, self.cache = pts, q, top, {}

    def __getitem__(self, v):
        if v not in self.cache:
            self.cache[v] = powers_of(cx_from_dd(self.pts[v, self.q]), self.top)
        return self.cache[v]


def evaluate_point(system, pts, q: int, polys=None):
    """Exact f_p and row J[p, :] at point index q of ``pts`` (float64 [n, P, 4]
    or, for quad-double points, [n, P, 8]).

    Returns (f, J): f[p] an exact complex; J[p] a dict {i: exact complex} of
    the variables that occur in polynomial p (absent entries are exactly 0).
    ``polys`` restricts the work to a subset of polynomial indices."""
    top = system.max_exp
    pw = _LazyPowers(pts, q, top)
    coefs = system.coef
    f, J = {}, {}
    for p in (range(system.n_polys) if polys is None else polys):
        fp = ZERO
        Jp = {}
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            pos, exp = system.monomial(t)
            c = cx_from_dd(coefs[t])
            # value term: c * prod_j x_{i_j}^{a_j}
            term = c
            for v, a in zip(pos, exp):
                term = cx_mul(term, pw[v][a])
            fp = cx_add(fp, term)
            # derivative terms: c * a_i * x_i^{a_i - 1} * prod_{j != i} x_j^{a_j}
            for i, ai in zip(pos, exp):
                d = cx_scale(c, ai)
                for v, a in zip(pos, exp):
                    d = cx_mul(d, pw[v][a - 1] if v == i else pw[v][a])
                Jp[i] = cx_add(Jp.get(i, ZERO), d)
        f[p] = fp
        J[p] = Jp
    return f, J


def scales_point(system, pts, q: int, polys=None):
    """Normwise scales at point q: S_f[p] = sum |c| |x|^a and
    S_J[p][i] = sum |c| a_i |x_i|^(a_i - 1) prod_{j != i} |x_j|^{a_j}, in float64."""
    wp = pts.shape[-1] // 2  # leading part of the imaginary component
    wc = system.coef.shape[-1] // 2
    ax = {}
    for v in set(system.pos.tolist()):
        ax[v] = math.hypot(pts[v, q, 0], pts[v, q, wp])
    Sf, SJ = {}, {}
    for p in (range(system.n_polys) if polys is None else polys):
        sf = 0.0
        sj = {}
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            pos, exp = system.monomial(t)
            ac = math.hypot(system.coef[t, 0], system.coef[t, wc])
            term = ac
            for v, a in zip(pos, exp):
                term *= ax[v] ** a
            sf += term
            for i, ai in zip(pos, exp):
                d = ac * ai
                for v, a in zip(pos, exp):
                    d *= ax[v] ** (a - 1 if v == i else a)
                sj[i] = sj.get(i, 0.0) + d
        Sf[p] = sf
        SJ[p] = sj
    return Sf, SJ


def normwise_error(got: Sequence[float], exact, scale: float) -> float:
    """|got - exact| / scale; got is a complex double-double (4 floats) or
    quad-double (8 floats).
    When the scale is 0 (no term contributes) the value must be exactly 0:
    returns 0 if it is and inf otherwise."""
    if not all(math.isfinite(v) for v in got):
        return math.inf
    diff = cx_sub(cx_from_dd(got), exact)
    if scale == 0.0:
        return 0.0 if (diff[0] == 0 and diff[1] == 0) else math.inf
    return cx_abs(diff) / scale


def max_errors(system, pts, out_f, out_J, points_idx: Sequence[int], polys=None):
    """Largest normwise errors (f, J) of computed outputs at the given points.

    out_f: float64 [N, P, c]; out_J: float64 [N, n, P, c] (structure of
    arrays, point-minor), c = 4 (double-double) or 8 (quad-double).  Entries J[p, i] for variables absent from
    polynomial p must be exactly zero."""
    ef = ej = 0.0
    n = system.n_vars
    for q in points_idx:
        f, J = evaluate_point(system, pts, q, polys)
        Sf, SJ = scales_point(system, pts, q, polys)
        for p in f:
            ef = max(ef, normwise_error(out_f[p, q], f[p], Sf[p]))
            for i in range(n):
                ex = J[p].get(i, ZERO)
                ej = max(ej, normwise_error(out_J[p, i, q], ex, SJ[p].get(i, 0.0)))
    return ef, ej


def evaluate_dd(system, pts, points_idx: Sequence[int]):
    """Exact results rounded to complex double-double, as arrays
    f [N, len(points_idx), 4] and J [N, n, len(points_idx), 4]."""
    import numpy as np

    N, n = system.n_polys, system.n_vars
    F = np.zeros((N, len(points_idx), 4))
    Jo = np.zeros((N, n, len(points_idx), 4))
    for c, q in enumerate(points_idx):
        f, J = evaluate_point(system, pts, q)
        for p in range(N):
            F[p, c] = cx_to_dd(f[p])
            for i, v in J[p].items():
                Jo[p, i, c] = cx_to_dd(v)
    return F, Jo
