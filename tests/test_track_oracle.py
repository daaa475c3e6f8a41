"""Pins for the path-tracking oracle (``oracle/track.py``), no GPU.

The tracker's end points are checked against solution sets reached another
way: the roots of a univariate polynomial from numpy's companion-matrix
eigenvalues, the product set of roots of a decoupled system, the solution of
a linear system from numpy's LU solver, and, for a generic dense system, the
residual of every end point by the exact oracle and the count of distinct
solutions (the Bezout number).
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import track as T


def match(found, want, tol):
    """Every wanted point has a distinct found point within tol (max norm)."""
    found = [np.asarray(f) for f in found]
    used = set()
    for w in want:
        d = [(np.max(np.abs(f - np.asarray(w))), i) for i, f in enumerate(found) if i not in used]
        best, i = min(d)
        if best > tol:
            return False
        used.add(i)
    return True


def test_univariate_roots_match_numpy():
    rng = np.random.Generator(np.random.PCG64(601))
    c = rng.standard_normal(6) + 1j * rng.standard_normal(6)  # degree 5, c[k] x^k
    mons = [([0], [k]) if k else ([], []) for k in range(6)]
    s = synth.from_monomials(1, [mons], [[z.real, 0, z.imag, 0] for z in c])
    res = T.solve_system(s)
    assert [st for _, st in res] == [T.SUCCESS] * 5
    assert match([x for x, _ in res], [[r] for r in np.roots(c[::-1])], 1e-9)


def test_decoupled_system_product_set():
    r0 = [0.5 + 0.25j, -1.0 + 0.5j]
    r1 = [1.5j, -0.75, 0.3 - 0.9j]
    def expand(roots, v):  # prod (x_v - r) as monomials of x_v
        c = np.array([1.0 + 0j])
        for r in roots:
            c = np.convolve(c, [1.0, -r])  # highest degree first
        deg = len(roots)
        mons, coef = [], []
        for k, a in enumerate(c):
            e = deg - k
            mons.append(([v], [e]) if e else ([], []))
            coef.append([a.real, 0, a.imag, 0])
        return mons, coef
    m0, c0 = expand(r0, 0)
    m1, c1 = expand(r1, 1)
    s = synth.from_monomials(2, [m0, m1], c0 + c1)
    res = T.solve_system(s)
    assert all(st == T.SUCCESS for _, st in res) and len(res) == 6
    assert match([x for x, _ in res], list(itertools.product(r0, r1)), 1e-9)


def test_linear_system_matches_numpy_solve():
    rng = np.random.Generator(np.random.PCG64(602))
    n = 3
    A = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    polys, coef = [], []
    for p in range(n):
        polys.append([([i], [1]) for i in range(n)] + [([], [])])
        coef += [[A[p, i].real, 0, A[p, i].imag, 0] for i in range(n)] + [[-b[p].real, 0, -b[p].imag, 0]]
    s = synth.from_monomials(n, polys, coef)
    (x, st), = T.solve_system(s)
    assert st == T.SUCCESS
    assert np.max(np.abs(np.asarray(x) - np.linalg.solve(A, b))) < 1e-12


def test_generic_dense_system_all_solutions():
    s = synth.dense_system(603, 2, [2, 3])
    res = T.solve_system(s)
    assert len(res) == 6 and all(st == T.SUCCESS for _, st in res)
    pts = np.zeros((2, len(res), 4))
    for q, (x, _) in enumerate(res):
        pts[:, q, 0] = [z.real for z in x]
        pts[:, q, 2] = [z.imag for z in x]
    for q in range(len(res)):
        f, _ = E.evaluate_point(s, pts, q)
        Sf, _ = E.scales_point(s, pts, q)
        for p in range(2):
            assert E.cx_abs(f[p]) <= 1e-12 * Sf[p]
    X = np.array([x for x, _ in res])
    d = np.abs(X[:, None, :] - X[None, :, :]).max(axis=2) + np.eye(len(res))
    assert d.min() > 1e-6  # distinct


def test_start_points_are_roots_of_unity_in_mixed_radix_order():
    pts = T.start_points([2, 3])
    assert len(pts) == 6
    for r, x in enumerate(pts):
        k0, k1 = r % 2, (r // 2) % 3
        assert abs(x[0] - np.exp(2j * np.pi * k0 / 2)) < 1e-15
        assert abs(x[1] - np.exp(2j * np.pi * k1 / 3)) < 1e-15


def test_no_finite_solutions_paths_do_not_succeed():
    # x y - 1 = 0 and x y - 2 = 0 have no solution: every path leaves for infinity
    s = synth.from_monomials(2, [[([0, 1], [1, 1]), ([], [])], [([0, 1], [1, 1]), ([], [])]],
                             [[1, 0, 0, 0], [-1, 0, 0, 0], [1, 0, 0, 0], [-2, 0, 0, 0]])
    res = T.solve_system(s, T.Params(max_steps=5000))
    assert all(st != T.SUCCESS for _, st in res)


def _track_pins():
    return [test_univariate_roots_match_numpy, test_decoupled_system_product_set,
            test_linear_system_matches_numpy_solve, test_start_points_are_roots_of_unity_in_mixed_radix_order]


def _mistake(name, monkeypatch):
    eval_fJ, solve, start = T.eval_fJ, T.solve, T.start_points
    if name == "jacobian_transposed":
        def wrong(system, x):
            F, J = eval_fJ(system, x)
            return F, [list(r) for r in zip(*J)]
        monkeypatch.setattr(T, "eval_fJ", wrong)
    elif name == "dropped_last_term":
        def wrong(system, x):
            F, J = eval_fJ(system, x)
            return [f - (1 if i == len(F) - 1 else 0) for i, f in enumerate(F)], J
        monkeypatch.setattr(T, "eval_fJ", wrong)
    elif name == "negated_solution":
        monkeypatch.setattr(T, "solve", lambda A, b: None if solve(A, b) is None else [-y for y in solve(A, b)])
    elif name == "start_points_off_the_roots_of_unity":
        monkeypatch.setattr(T, "start_points", lambda degs: [[1.1 * z for z in x] for x in start(degs)])


@pytest.mark.parametrize("name", ["jacobian_transposed", "dropped_last_term", "negated_solution",
                                  "start_points_off_the_roots_of_unity"])
def test_planted_mistake_in_the_tracking_oracle_is_caught(name, monkeypatch):
    """A mistake planted in the tracking oracle fails at least one pin."""
    _mistake(name, monkeypatch)
    results = []
    for pin in _track_pins():
        try:
            pin()
            results.append(True)
        except AssertionError:
            results.append(False)
    assert not all(results), f"{name} survived every pin"
