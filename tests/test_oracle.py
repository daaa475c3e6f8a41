"""Pins for the oracle, independent of the oracle itself.

Each check reaches the same numbers by another route than the power rule of
Section 2, Eq. (1) that ``oracle.exact`` writes out:

* forward-mode differentiation with dual numbers in ``fractions.Fraction``
  (monomials multiplied out factor by factor, no powers table, no power rule);
* linear systems f = A x + b, whose Jacobian is A (catches transposes and
  index mistakes) and whose value is a numpy matrix-vector product;
* Euler's identity sum_i x_i df/dx_i = d f on homogeneous systems;
* closed forms: c x^a and the Speelpenning product x_1 ... x_k;
* quad-double data: the dual-number route again with every coefficient and
  point a sum of four doubles whose lower two parts lie below double-double
  precision;
* brute force over all small monomials with Gaussian-integer data, the value
  from numpy and each derivative by exact Lagrange interpolation along the
  variable's line;
* planted mistakes (a sign, a dropped factor, a shifted power, a dropped term,
  a wrong index) in the oracle make at least one of the checks fail.

The C double-double oracle is then pinned to the exact one.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import synth
from oracle import exact as E


# ----------------------------------------------------------------------------
# independent exact arithmetic: complex numbers as pairs of Fractions
# ----------------------------------------------------------------------------

def fr_from_dd(v):
    """A complex multi-double (2, 4 or 8 doubles: real parts, then imaginary
    parts) as a pair of Fractions."""
    w = len(v) // 2
    return (sum((Fraction(float(x)) for x in v[:w]), Fraction(0)),
            sum((Fraction(float(x)) for x in v[w:2 * w]), Fraction(0)))


def fr_from_exact(z):
    a, b, e = z
    s = Fraction(2) ** e
    return (a * s, b * s)


def fmul(x, y):
    return (x[0] * y[0] - x[1] * y[1], x[0] * y[1] + x[1] * y[0])


def fadd(x, y):
    return (x[0] + y[0], x[1] + y[1])


FZERO = (Fraction(0), Fraction(0))
FONE = (Fraction(1), Fraction(0))


def dual_mul(u, v):
    """(a + eps b)(c + eps d) = ac + eps (ad + bc), eps^2 = 0."""
    return (fmul(u[0], v[0]), fadd(fmul(u[0], v[1]), fmul(u[1], v[0])))


def dual_eval(system, pts, q, direction):
    """f_p(x + eps e_direction) for every p; returns [(value, eps-part)]."""
    n = system.n_vars
    xs = []
    for v in range(n):
        xv = fr_from_dd(pts[v, q])
        xs.append((xv, FONE if v == direction else FZERO))
    out = []
    for p in range(system.n_polys):
        acc = (FZERO, FZERO)
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            pos, exp = system.monomial(t)
            term = (fr_from_dd(system.coef[t]), FZERO)
            for v, a in zip(pos, exp):
                for _ in range(a):
                    term = dual_mul(term, xs[v])
            acc = (fadd(acc[0], term[0]), fadd(acc[1], term[1]))
        out.append(acc)
    return out


def random_dd_system(seed, n, N, m, kmax, emax, allow_k0=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _p in range(N):
        mons = []
        for _t in range(m):
            k = int(rng.integers(0 if allow_k0 else 1, kmax + 1))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            exp = rng.integers(1, emax + 1, size=k).tolist()
            mons.append((pos, exp))
        polys.append(mons)
    coef = synth.random_cdd(rng, N * m)
    return synth.from_monomials(n, polys, coef)


# ----------------------------------------------------------------------------
# the checks (functions so the mutation test can rerun them)
# ----------------------------------------------------------------------------

def check_dual(seed=1):
    s = random_dd_system(seed, n=4, N=3, m=5, kmax=3, emax=3)
    pts = synth.points(seed + 7, 4, 2)
    for q in range(2):
        f, J = E.evaluate_point(s, pts, q)
        for i in range(s.n_vars):
            ref = dual_eval(s, pts, q, i)
            for p in range(s.n_polys):
                if fr_from_exact(f[p]) != ref[p][0]:
                    return False
                if fr_from_exact(J[p].get(i, E.ZERO)) != ref[p][1]:
                    return False
    return True


def check_linear(seed=2):
    rng = np.random.Generator(np.random.PCG64(seed))
    N, n = 3, 5
    A = rng.integers(-4, 5, size=(N, n)) + 1j * rng.integers(-4, 5, size=(N, n))
    A[rng.random((N, n)) < 0.3] = 0
    b = rng.integers(-4, 5, size=N) + 1j * rng.integers(-4, 5, size=N)
    polys, coef = [], []
    for p in range(N):
        mons = []
        for i in range(n):
            if A[p, i] != 0:
                mons.append(([i], [1]))
                coef.append([A[p, i].real, 0, A[p, i].imag, 0])
        mons.append(([], []))
        coef.append([b[p].real, 0, b[p].imag, 0])
        polys.append(mons)
    s = synth.from_monomials(n, polys, coef)
    xs = rng.integers(-3, 4, size=n) + 1j * rng.integers(-3, 4, size=n)
    pts = np.zeros((n, 1, 4))
    pts[:, 0, 0] = xs.real
    pts[:, 0, 2] = xs.imag
    f, J = E.evaluate_point(s, pts, 0)
    fv = A @ xs + b  # small Gaussian integers: exact in complex128
    for p in range(N):
        if fr_from_exact(f[p]) != (Fraction(fv[p].real), Fraction(fv[p].imag)):
            return False
        for i in range(n):
            if fr_from_exact(J[p].get(i, E.ZERO)) != (Fraction(A[p, i].real), Fraction(A[p, i].imag)):
                return False
    return True


def check_euler(seed=3):
    deg = 7
    rng = np.random.Generator(np.random.PCG64(seed))
    n, N, m = 5, 3, 6
    polys = []
    for _p in range(N):
        mons = []
        for _t in range(m):
            k = int(rng.integers(1, 5))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            exp = [1] * k
            for _u in range(deg - k):
                exp[int(rng.integers(0, k))] += 1
            mons.append((pos, exp))
        polys.append(mons)
    s = synth.from_monomials(n, polys, synth.random_cdd(rng, N * m))
    pts = synth.points(seed + 11, n, 2, modulus_octaves=(-1, 0))
    for q in range(2):
        f, J = E.evaluate_point(s, pts, q)
        for p in range(N):
            lhs = FZERO
            for i in range(n):
                lhs = fadd(lhs, fmul(fr_from_dd(pts[i, q]), fr_from_exact(J[p].get(i, E.ZERO))))
            fp = fr_from_exact(f[p])
            if lhs != (deg * fp[0], deg * fp[1]):
                return False
    return True


def check_closed_forms(seed=4):
    rng = np.random.Generator(np.random.PCG64(seed))
    # c x^a: f = c x^a, f' = a c x^(a-1)
    for a in range(1, 7):
        c = complex(int(rng.integers(-3, 4)), int(rng.integers(1, 4)))
        x = complex(int(rng.integers(-2, 3)), int(rng.integers(-2, 3)))
        s = synth.from_monomials(1, [[([0], [a])]], [[c.real, 0, c.imag, 0]])
        pts = np.array([[[x.real, 0, x.imag, 0]]])
        f, J = E.evaluate_point(s, pts, 0)
        fv = c * x ** a
        dv = a * c * x ** (a - 1)
        if fr_from_exact(f[0]) != (Fraction(fv.real), Fraction(fv.imag)):
            return False
        if fr_from_exact(J[0][0]) != (Fraction(dv.real), Fraction(dv.imag)):
            return False
    # Speelpenning: d/dx_i (x_1 ... x_k) = prod_{j != i} x_j
    k = 6
    xs = [complex(int(rng.integers(-2, 3)), int(rng.integers(-2, 3))) for _ in range(k)]
    s = synth.from_monomials(k, [[(list(range(k)), [1] * k)]], [[1, 0, 0, 0]])
    pts = np.zeros((k, 1, 4))
    pts[:, 0, 0] = [z.real for z in xs]
    pts[:, 0, 2] = [z.imag for z in xs]
    f, J = E.evaluate_point(s, pts, 0)
    if fr_from_exact(f[0]) != (Fraction(math.prod(xs).real), Fraction(math.prod(xs).imag)):
        return False
    for i in range(k):
        d = math.prod(xs[:i] + xs[i + 1:])
        if fr_from_exact(J[0][i]) != (Fraction(d.real), Fraction(d.imag)):
            return False
    return True


def lagrange_derivative(samples, t0):
    """Derivative at t0 of the polynomial through (t, y) samples, exactly.
    y are complex pairs of Fractions."""
    res = FZERO
    ts = [t for t, _ in samples]
    for j, (tj, yj) in enumerate(samples):
        # d/dt L_j(t) at t0 = sum_{m != j} prod_{l != j, m} (t0 - t_l) / prod_{l != j} (tj - t_l)
        den = Fraction(1)
        for l, tl in enumerate(ts):
            if l != j:
                den *= (tj - tl)
        num = Fraction(0)
        for mm, tm in enumerate(ts):
            if mm == j:
                continue
            pr = Fraction(1)
            for l, tl in enumerate(ts):
                if l != j and l != mm:
                    pr *= (t0 - tl)
            num += pr
        w = num / den
        res = fadd(res, (yj[0] * w, yj[1] * w))
    return res


def check_brute_force(seed=5):
    """Every monomial in 2 variables with exponents <= 2 (and the constant),
    Gaussian-integer coefficients; every point of a Gaussian-integer grid."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n = 2
    mons = []
    for e0 in range(3):
        for e1 in range(3):
            pos = [v for v, e in ((0, e0), (1, e1)) if e > 0]
            exp = [e for e in (e0, e1) if e > 0]
            mons.append((pos, exp))
    coef = synth.gaussian_int_cdd(rng, len(mons))
    s = synth.from_monomials(n, [mons], coef)
    grid = [complex(a, b) for a in (-2, 0, 1) for b in (-1, 2)]
    c = coef[:, 0] + 1j * coef[:, 2]
    for x0, x1 in itertools.product(grid, grid):
        pts = np.array([[[x0.real, 0, x0.imag, 0]], [[x1.real, 0, x1.imag, 0]]])
        f, J = E.evaluate_point(s, pts, 0)
        # value by numpy: sum c * x0^e0 * x1^e1 (exact for these small integers)
        fv = 0
        for (pos, exp), cc in zip(mons, c):
            term = cc
            for v, a in zip(pos, exp):
                term = term * np.power((x0, x1)[v], a)
            fv += term
        if fr_from_exact(f[0]) != (Fraction(fv.real), Fraction(fv.imag)):
            return False
        # derivatives by exact interpolation along each variable's line
        for i in range(n):
            samples = []
            for tt in range(5):
                xx = [x0, x1]
                xx[i] = xx[i] + tt
                val = FZERO
                for (pos, exp), cc in zip(mons, coef):
                    term = fr_from_dd(cc)
                    for v, a in zip(pos, exp):
                        xv = (Fraction(xx[v].real), Fraction(xx[v].imag))
                        for _ in range(a):
                            term = fmul(term, xv)
                    val = fadd(val, term)
                samples.append((Fraction(tt), val))
            if fr_from_exact(J[0].get(i, E.ZERO)) != lagrange_derivative(samples, Fraction(0)):
                return False
    return True


def check_quad_double(seed=6):
    """Dual numbers over quad-double coefficients and points."""
    s = random_dd_system(seed, n=4, N=3, m=5, kmax=3, emax=3).to_qd(seed + 1)
    rng = np.random.Generator(np.random.PCG64(seed + 2))
    pts = synth.widen_qd(rng, synth.points(seed + 7, 4, 2))
    # the lower parts matter: dropping them changes the data
    assert any(fr_from_dd(c) != fr_from_dd(c[[0, 1, 4, 5]]) for c in s.coef)
    for q in range(2):
        f, J = E.evaluate_point(s, pts, q)
        for i in range(s.n_vars):
            ref = dual_eval(s, pts, q, i)
            for p in range(s.n_polys):
                if fr_from_exact(f[p]) != ref[p][0]:
                    return False
                if fr_from_exact(J[p].get(i, E.ZERO)) != ref[p][1]:
                    return False
    return True


CHECKS = [check_dual, check_linear, check_euler, check_closed_forms, check_brute_force, check_quad_double]


@pytest.mark.parametrize("check", CHECKS, ids=lambda c: c.__name__)
def test_oracle_pin(check):
    assert check()


# ----------------------------------------------------------------------------
# planted mistakes must be caught
# ----------------------------------------------------------------------------

def _mut_sign(x, y):
    a, b, e = x
    c, d, f = y
    return (a * c - b * d, a * d - b * c, e + f)


def _mut_scale(x, k):
    return x


_orig_powers = E.powers_of


def _mut_powers(xv, top):
    p = _orig_powers(xv, top + 1)
    return p[1:]


_orig_add = E.cx_add


class _DropEvery3:
    def __init__(self):
        self.i = 0

    def __call__(self, x, y):
        self.i += 1
        return x if self.i % 3 == 0 else _orig_add(x, y)


_orig_monomial = synth.System.monomial


def _mut_index(self, t):
    pos, exp = _orig_monomial(self, t)
    if len(pos) >= 2:
        pos = [pos[1], pos[0]] + pos[2:]
    return pos, exp


_orig_from_dd = E.cx_from_dd


def _mut_two_parts(v):
    """Reads only the leading two parts of each component."""
    w = len(v) // 2
    return _orig_from_dd([v[0], v[1], v[w], v[w + 1]])


MUTATIONS = {
    "quad_double_low_parts_dropped": (E, "cx_from_dd", _mut_two_parts),
    "wrong_sign": (E, "cx_mul", _mut_sign),
    "dropped_exponent_factor": (E, "cx_scale", _mut_scale),
    "power_off_by_one": (E, "powers_of", _mut_powers),
    "dropped_term": (E, "cx_add", None),
    "swapped_index": (synth.System, "monomial", _mut_index),
}


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(name, monkeypatch):
    obj, attr, fn = MUTATIONS[name]
    if fn is None:
        fn = _DropEvery3()
    monkeypatch.setattr(obj, attr, fn)
    results = []
    for check in CHECKS:
        try:
            results.append(check())
        except Exception:
            results.append(False)
    assert not all(results), f"mutation {name} survived every pin"


# ----------------------------------------------------------------------------
# exact helpers
# ----------------------------------------------------------------------------

def test_qd_rounding_round_trip_and_bound():
    """A normalised quad-double is its own rounding; rounding an exact value
    to quad-double errs by at most 2^-211 of it (four parts of 53 bits, each
    rounded to nearest); the parts are normalised."""
    rng = np.random.Generator(np.random.PCG64(31))
    vals = synth.widen_qd(rng, synth.random_cdd(rng, 50))
    for v in vals:
        assert E.cx_to_qd(E.cx_from_dd(v)) == tuple(float(x) for x in v)
    for i in range(50):
        # an exact product of three quad-doubles needs about 640 bits
        z = E.cx_mul(E.cx_mul(E.cx_from_dd(vals[i]), E.cx_from_dd(vals[(i + 1) % 50])), E.cx_from_dd(vals[(i + 2) % 50]))
        r = E.cx_to_qd(z)
        err = E.cx_abs(E.cx_sub(E.cx_from_dd(r), z))
        assert err <= 2.0 ** -211 * E.cx_abs(z)
        for c in (0, 4):
            for k in range(3):
                hi, lo = r[c + k], r[c + k + 1]
                assert abs(lo) <= math.ulp(hi) / 2 or hi == 0.0


def test_dd_round_trip_and_rounding():
    rng = np.random.Generator(np.random.PCG64(9))
    v = synth.random_cdd(rng, 200)
    for row in v:
        z = E.cx_from_dd(row)
        back = E.cx_to_dd(z)
        assert tuple(back) == tuple(row)
    # a value needing more than 106 bits rounds to nearest hi, then lo
    z = ((1 << 120) + 3, 0, -120)
    hi, lo, _, _ = E.cx_to_dd(z)
    assert hi == 1.0 and lo == 3 * 2.0 ** -120


def test_normwise_error_zero_scale_requires_exact_zero():
    assert E.normwise_error((0.0, 0.0, 0.0, 0.0), E.ZERO, 0.0) == 0.0
    assert E.normwise_error((1e-300, 0.0, 0.0, 0.0), E.ZERO, 0.0) == math.inf
    assert E.normwise_error((float("nan"), 0.0, 0.0, 0.0), E.ZERO, 1.0) == math.inf


# ----------------------------------------------------------------------------
# the C double-double oracle against the exact one
# ----------------------------------------------------------------------------

def test_c_dd_oracle_exact_on_gaussian_integers():
    import oracle

    rng = np.random.Generator(np.random.PCG64(21))
    n = 4
    polys = []
    for _p in range(3):
        mons = []
        for _t in range(6):
            k = int(rng.integers(0, 4))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, 4, size=k).tolist()))
        polys.append(mons)
    s = synth.from_monomials(n, polys, synth.gaussian_int_cdd(rng, 18))
    pts = np.zeros((n, 5, 4))
    pts[:, :, 0] = rng.integers(-2, 3, size=(n, 5))
    pts[:, :, 2] = rng.integers(-2, 3, size=(n, 5))
    F, J = oracle.dd_eval(s, pts, threads=2)
    Fx, Jx = E.evaluate_dd(s, pts, range(5))
    assert np.array_equal(F, Fx)
    assert np.array_equal(J, Jx)


@pytest.mark.parametrize("cfg", [1, 2])
def test_c_dd_oracle_within_dd_tolerance(cfg):
    import oracle

    s, pts = synth.config(cfg, n_points=3)
    F, J = oracle.dd_eval(s, pts, threads=2)
    polys = None if cfg == 1 else [0, 17, 31]
    ef, ej = E.max_errors(s, pts, F, J, range(pts.shape[1]), polys=polys)
    assert ef <= 1e-30 and ej <= 1e-30, (ef, ej)


@pytest.mark.parametrize("cfg", [3, 5])
def test_c_dd_oracle_within_dd_tolerance_on_large_shapes(cfg):
    """The dense GPU samples of the n = 64 and n = 128 workloads are compared
    with the C oracle; here the C oracle itself is held to 1e-30 of the exact
    values (Section 2, Eq. 1) on the first and last polynomial at one point of
    those shapes (k = 16 and 32, exponents up to 8 and 4)."""
    import oracle

    s, pts = synth.config(cfg, n_points=1)
    F, J = oracle.dd_eval(s, pts, threads=2)
    ef, ej = E.max_errors(s, pts, F, J, range(1), polys=[0, s.n_polys - 1])
    assert ef <= 1e-30 and ej <= 1e-30, (ef, ej)


def test_c_dd_oracle_point_range_and_args():
    import oracle

    s, pts = synth.config(1, n_points=4)
    F, J = oracle.dd_eval(s, pts, q0=1, q1=3)
    assert np.all(F[:, 0] == 0) and np.all(F[:, 3] == 0)
    assert np.any(F[:, 1] != 0)
    with pytest.raises(ValueError):
        oracle.dd_eval(s, pts, q0=3, q1=2)


# ----------------------------------------------------------------------------
# the exact Newton step
# ----------------------------------------------------------------------------

def test_newton_exact_on_linear_system_lands_on_solution():
    """f = A x - b: one Newton step from any x0 gives A x1 = b (checked by a
    plain matrix-vector product)."""
    from oracle import newton as N

    rng = np.random.Generator(np.random.PCG64(31))
    n = 4
    A = rng.integers(-3, 4, size=(n, n)) + 1j * rng.integers(-3, 4, size=(n, n)) + 5 * np.eye(n)
    b = rng.integers(-3, 4, size=n) + 1j * rng.integers(-3, 4, size=n)
    polys, coef = [], []
    for p in range(n):
        mons = [([i], [1]) for i in range(n) if A[p, i] != 0] + [([], [])]
        coef += [[A[p, i].real, 0, A[p, i].imag, 0] for i in range(n) if A[p, i] != 0]
        coef.append([-b[p].real, 0, -b[p].imag, 0])
        polys.append(mons)
    s = synth.from_monomials(n, polys, coef)
    pts = synth.points(32, n, 1)
    _f, _J, _dx, x1 = N.newton_step(s, pts, 0)
    for p in range(n):
        acc = N.ZERO
        for i in range(n):
            acc = N.c_add(acc, N.c_mul((Fraction(A[p, i].real), Fraction(A[p, i].imag)), x1[i]))
        assert acc == (Fraction(b[p].real), Fraction(b[p].imag))


def test_newton_exact_univariate_closed_form():
    """f = x^2 - c: x1 = (x0^2 + c) / (2 x0)."""
    from oracle import newton as N

    c = complex(2, 1)
    s = synth.from_monomials(1, [[([0], [2]), ([], [])]], [[1, 0, 0, 0], [-c.real, 0, -c.imag, 0]])
    pts = np.array([[[1.5, 0, 0.25, 0]]])
    _f, _J, _dx, x1 = N.newton_step(s, pts, 0)
    x0 = (Fraction(1.5), Fraction(0.25))
    want = N.c_div(N.c_add(N.c_mul(x0, x0), (Fraction(2), Fraction(1))), N.c_mul((Fraction(2), Fraction(0)), x0))
    assert x1[0] == want


def test_newton_exact_residual_identity():
    """J dx = -f exactly for a random square system."""
    from oracle import newton as N

    s = random_dd_system(33, n=3, N=3, m=4, kmax=3, emax=3, allow_k0=True)
    pts = synth.points(34, 3, 2)
    for q in range(2):
        f, J, dx, _ = N.newton_step(s, pts, q)
        for i in range(3):
            acc = f[i]
            for j in range(3):
                acc = N.c_add(acc, N.c_mul(J[i][j], dx[j]))
            assert acc == N.ZERO


def _newton_pins():
    return [test_newton_exact_on_linear_system_lands_on_solution, test_newton_exact_univariate_closed_form,
            test_newton_exact_residual_identity]


@pytest.mark.parametrize("mistake", ["negated_step", "transposed_jacobian", "wrong_division", "dropped_pivot_row"])
def test_newton_planted_mistake_is_caught(mistake, monkeypatch):
    """A plausible mistake planted in the Newton oracle's solve fails at least
    one of the Newton pins above."""
    from oracle import newton as N

    solve, c_div = N.solve, N.c_div
    if mistake == "negated_step":
        monkeypatch.setattr(N, "solve", lambda A, b: [(-x[0], -x[1]) for x in solve(A, b)])
    elif mistake == "transposed_jacobian":
        monkeypatch.setattr(N, "solve", lambda A, b: solve([list(r) for r in zip(*A)], b))
    elif mistake == "wrong_division":  # conjugate of the right quotient
        monkeypatch.setattr(N, "c_div", lambda x, y: (c_div(x, y)[0], -c_div(x, y)[1]))
    else:  # elimination that skips the last row
        def partial(A, b):
            n = len(A)
            if n == 1:
                return solve(A, b)
            x = solve([row[:n - 1] for row in A[:n - 1]], b[:n - 1])
            return x + [N.ZERO]
        monkeypatch.setattr(N, "solve", partial)
    results = []
    for pin in _newton_pins():
        try:
            pin()
            results.append(True)
        except AssertionError:
            results.append(False)
    assert not all(results), f"{mistake} survived every Newton pin"
