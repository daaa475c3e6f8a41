"""Exact Newton step -- TEST INFRASTRUCTURE ONLY (only tests/ use it).

Newton's method is the corrector the paper's evaluation serves (Section 1):
from x0, the step dx solves J(x0) dx = -f(x0) and x1 = x0 + dx.  Here f and J
come from the exact oracle (``oracle.exact``, Section 2, Eq. 1) and the linear
system is solved exactly by Gaussian elimination over the complex rationals
(pairs of ``fractions.Fraction``), so x1 is the exact Newton iterate.
"""
from __future__ import annotations

from fractions import Fraction

from . import exact as E


def fr(z):
    """An exact complex dyadic (A, B, e) as a pair of Fractions."""
    a, b, e = z
    s = Fraction(2) ** e
    return (a * s, b * s)


def c_add(x, y):
    return (x[0] + y[0], x[1] + y[1])


def c_sub(x, y):
    return (x[0] - y[0], x[1] - y[1])


def c_mul(x, y):
    return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])


def c_div(x, y):
    d = y[0] * y[0] + y[1] * y[1]
    return ((x[0] * y[0] + x[1] * y[1]) / d, (x[1] * y[0] - x[0] * y[1]) / d)


ZERO = (Fraction(0), Fraction(0))


def solve(A, b):
    """x with A x = b, by Gaussian elimination (any nonzero pivot: the
    arithmetic is exact).  A: list of rows of complex pairs; raises
    ZeroDivisionError for a singular A."""
    n = len(A)
    M = [list(row) + [b[i]] for i, row in enumerate(A)]
    for k in range(n):
        piv = next((i for i in range(k, n) if M[i][k] != ZERO), None)
        if piv is None:
            raise ZeroDivisionError("singular matrix")
        M[k], M[piv] = M[piv], M[k]
        for i in range(k + 1, n):
            if M[i][k] == ZERO:
                continue
            l = c_div(M[i][k], M[k][k])
            for j in range(k, n + 1):
                M[i][j] = c_sub(M[i][j], c_mul(l, M[k][j]))
    x = [ZERO] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n]
        for j in range(i + 1, n):
            s = c_sub(s, c_mul(M[i][j], x[j]))
        x[i] = c_div(s, M[i][i])
    return x


def f_and_J(system, pts, q):
    """Exact f and J at point q of ``pts`` (float64 [n, P, 4] or [n, P, 8])
    of a square system, as complex Fraction pairs (f[i], J[i][j])."""
    n = system.n_vars
    if system.n_polys != n:
        raise ValueError("Newton's method needs a square system")
    fe, Je = E.evaluate_point(system, pts, q)
    f = [fr(fe[i]) for i in range(n)]
    J = [[fr(Je[i].get(j, E.ZERO)) for j in range(n)] for i in range(n)]
    return f, J


def newton_step(system, pts, q):
    """Exact (f, J, dx, x1) at point q of ``pts`` (float64 [n, P, 4] or
    [n, P, 8]) for a square system: f and J as in ``f_and_J``."""
    n = system.n_vars
    f, J = f_and_J(system, pts, q)
    dx = solve(J, [c_sub(ZERO, fi) for fi in f])
    x0 = [fr(E.cx_from_dd(pts[v, q])) for v in range(n)]
    return f, J, dx, [c_add(x0[i], dx[i]) for i in range(n)]
