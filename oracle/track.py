"""Path tracking oracle.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this module;
only ``tests/`` may use it.

The application the paper evaluates f and J for (Section 1): solving a
square polynomial system F(x) = 0 by homotopy continuation, with Newton's
method as the corrector of a path tracker.  This is a plain, slow tracker in
Python complex arithmetic (double precision), one path at a time:

* homotopy H(x, t) = gamma (1 - t) G(x) + t F(x) with G_i(x) = x_i^(d_i) - 1,
  d_i the total degree of polynomial i (the total-degree homotopy with the
  "gamma trick");
* start solutions: every vector of roots of unity (x_i^(d_i) = 1), in
  mixed-radix order of the path index (radices d_0, d_1, ...);
* predictor: an Euler step along the tangent, H_x v = -H_t with
  H_t = F - gamma G;
* corrector: Newton's method on H(., t1); a step is accepted when
  max|dx| <= corr_tol max(1, max|x|) within max_corr iterations whose steps
  shrink; otherwise the path goes back to its last accepted point and the
  step size is halved (the path fails below h_min); after succ_grow accepted
  steps in a row the step size doubles, up to h_max;
* at t = 1: Newton's method on F until max|dx| <= end_tol max(1, max|x|).

F and J_F are evaluated from the definitions of Section 2, Eq. (1), term by
term, and the linear systems are solved by Gaussian elimination with partial
pivoting written out below.
"""
from __future__ import annotations

import cmath
import math
from dataclasses import dataclass
from typing import List, Sequence, Tuple

RUNNING, SUCCESS, FAILED, DIVERGED, END_NOT_CONVERGED = 0, 1, 2, 3, 4


@dataclass
class Params:
    gamma: complex = complex(math.cos(1.0), math.sin(1.0))
    h_init: float = 0.02
    h_min: float = 1e-10
    h_max: float = 0.1
    corr_tol: float = 1e-9
    end_tol: float = 1e-13
    x_big: float = 1e8
    max_corr: int = 3
    max_end: int = 8
    succ_grow: int = 3
    max_steps: int = 100000


def _complex(v: Sequence[float]) -> complex:
    """Leading parts of a complex multi-double (re, ..., im, ...)."""
    w = len(v) // 2
    return complex(float(v[0]), float(v[w]))


def degrees(system) -> List[int]:
    out = []
    for p in range(system.n_polys):
        d = 0
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            d = max(d, sum(system.monomial(t)[1]))
        out.append(d)
    return out


def eval_fJ(system, x: Sequence[complex]):
    """F(x) and J_F(x) by the definitions (Section 2, Eq. 1)."""
    n, N = system.n_vars, system.n_polys
    F = [0j] * N
    J = [[0j] * n for _ in range(N)]
    for p in range(N):
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            pos, exp = system.monomial(t)
            c = _complex(system.coef[t])
            term = c
            for v, a in zip(pos, exp):
                term *= x[v] ** a
            F[p] += term
            for i, ai in zip(pos, exp):
                d = c * ai
                for v, a in zip(pos, exp):
                    d *= x[v] ** (a - 1) if v == i else x[v] ** a
                J[p][i] += d
    return F, J


def solve(A, b):
    """A y = b by Gaussian elimination with partial pivoting; None if a pivot
    column is exactly zero."""
    n = len(b)
    M = [list(A[i]) + [b[i]] for i in range(n)]
    for k in range(n):
        piv = max(range(k, n), key=lambda i: abs(M[i][k]))
        if M[piv][k] == 0:
            return None
        M[k], M[piv] = M[piv], M[k]
        for i in range(k + 1, n):
            l = M[i][k] / M[k][k]
            for j in range(k, n + 1):
                M[i][j] -= l * M[k][j]
    y = [0j] * n
    for i in range(n - 1, -1, -1):
        s = M[i][n] - sum(M[i][j] * y[j] for j in range(i + 1, n))
        y[i] = s / M[i][i]
    return y


def start_points(degs: Sequence[int]) -> List[List[complex]]:
    """All start solutions, path r with the mixed-radix digits of r."""
    total = math.prod(degs)
    out = []
    for r in range(total):
        x = []
        for d in degs:
            k = r % d
            r //= d
            x.append(cmath.exp(2j * math.pi * k / d))
        out.append(x)
    return out


def _homotopy(system, degs, gamma, x, t):
    """H_x, H and H_t at (x, t)."""
    F, JF = eval_fJ(system, x)
    n = len(x)
    G = [x[i] ** degs[i] - 1 for i in range(n)]
    a = gamma * (1 - t)
    Hx = [[t * JF[i][j] for j in range(n)] for i in range(n)]
    for i in range(n):
        Hx[i][i] += a * degs[i] * x[i] ** (degs[i] - 1)
    H = [a * G[i] + t * F[i] for i in range(n)]
    Ht = [F[i] - gamma * G[i] for i in range(n)]
    return Hx, H, Ht


def track_path(system, x0: Sequence[complex], prm: Params = Params()) -> Tuple[List[complex], int, float]:
    """One path from t = 0 (x0) to t = 1: (end point, status, last t)."""
    degs = degrees(system)
    n = len(x0)
    x = list(x0)
    xs = list(x0)
    t, t1, h = 0.0, 0.0, prm.h_init
    phase, it, succ, dprev = "correct", 0, 0, math.inf
    for _ in range(prm.max_steps):
        tt = t if phase == "predict" else (1.0 if phase == "end" else t1)
        Hx, H, Ht = _homotopy(system, degs, prm.gamma, x, tt)
        rhs = [-v for v in Ht] if phase == "predict" else [-v for v in H]
        y = solve(Hx, rhs)
        if y is None:
            if phase == "end":
                return x, END_NOT_CONVERGED, t
            x, h, succ, it, phase = list(xs), h / 2, 0, 0, "predict"
            if h < prm.h_min:
                return x, FAILED, t
            continue
        if phase == "predict":
            t1 = min(t + h, 1.0)
            x = [x[i] + (t1 - t) * y[i] for i in range(n)]
            phase, it, dprev = "correct", 0, math.inf
            continue
        x = [x[i] + y[i] for i in range(n)]
        dxn = max(abs(v) for v in y)
        xn = max(abs(v) for v in x)
        it += 1
        scale = max(1.0, xn)
        if not xn <= prm.x_big:
            return x, DIVERGED, t
        if phase == "end":
            if dxn <= prm.end_tol * scale:
                return x, SUCCESS, t
            if it >= prm.max_end:
                return x, END_NOT_CONVERGED, t
        elif dxn <= prm.corr_tol * scale:
            t = t1
            xs = list(x)
            succ += 1
            if succ >= prm.succ_grow:
                h, succ = min(2 * h, prm.h_max), 0
            it = 0
            phase = "end" if t >= 1.0 else "predict"
        elif it >= prm.max_corr or (it >= 2 and dxn > dprev):
            x, h, succ, it, phase = list(xs), h / 2, 0, 0, "predict"
            if h < prm.h_min:
                return x, FAILED, t
        else:
            dprev = dxn
    return x, RUNNING, t


def solve_system(system, prm: Params = Params()):
    """Every path of the total-degree homotopy: [(end point, status)]."""
    return [track_path(system, x0, prm)[:2] for x0 in start_points(degrees(system))]
