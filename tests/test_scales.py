"""Pins for the normwise scales that every parity bar divides by.

S_f[p]    = sum_t |c_t| |x^{a_t}|
S_J[p][i] = sum_{t, i in t} |c_t| a_{t,i} |x_i|^{a_{t,i}-1} prod_{j != i} |x_j|^{a_{t,j}}

are the outputs f and J of a second polynomial system: the same monomials
with coefficients |c_t|, evaluated at the real point r = (|x_1|, ..., |x_n|)
(Section 2, Eq. 1 applied to moduli).  ``oracle.exact.scales_point`` and its
vectorised twin ``tests/_util.scales`` compute them in float64.  Nothing here
re-types their formula; each check reaches the numbers by another route:

* the exact oracle (itself pinned by dual numbers, Euler, brute force) on
  the moduli system at r;
* S_J as the gradient of S_f with respect to the moduli r_i (central
  differences of S_f along x_i -> (1 + h) x_i);
* Euler's identity sum_i r_i S_J[p][i] = d S_f[p] on a homogeneous system;
* exact powers of two for the Speelpenning product at points with |x_i| = 2^e_i;
* zero scales exactly where a variable is absent from a polynomial;
* the two implementations against each other on configs 1-3.

Planted mistakes (a dropped exponent factor, the exponent a_i where a_i - 1
belongs, a coefficient or point modulus taken from the real part only) make at
least one check fail, for both implementations.
"""
import math

import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import scales as vec_scales


def _point_fn(vectorised):
    """(system, pts, q) -> (S_f dict, S_J dict of dicts) for either implementation."""
    if not vectorised:
        return lambda s, pts, q: E.scales_point(s, pts, q)

    def fn(s, pts, q):
        Sf, SJ = vec_scales(s, np.ascontiguousarray(pts[:, q:q + 1]))
        f = {p: float(Sf[p, 0]) for p in range(s.n_polys)}
        J = {p: {i: float(SJ[p, i, 0]) for i in range(s.n_vars) if SJ[p, i, 0] != 0.0} for p in range(s.n_polys)}
        return f, J

    return fn


def _system(seed, n=6, N=4, m=7, kmax=4, emax=4, allow_k0=True):
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _p in range(N):
        mons = []
        for _t in range(m):
            k = int(rng.integers(0 if allow_k0 else 1, kmax + 1))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, emax + 1, size=k).tolist()))
        polys.append(mons)
    mod = np.ldexp(1.0 + rng.random(N * m), rng.integers(-3, 4, size=N * m))
    return synth.from_monomials(n, polys, synth.random_cdd(rng, N * m, mod))


def _moduli_system(s, pts, q):
    """The same monomials with coefficients |c| and the point |x| (leading
    parts, as the scales read them), as a system and a one-point array."""
    w = s.coef.shape[1] // 2
    c = np.zeros((s.n_monos, 4))
    c[:, 0] = [abs(complex(a, b)) for a, b in zip(s.coef[:, 0], s.coef[:, w])]
    ms = synth.System(s.n_vars, s.n_polys, s.poly_ptr, s.mono_ptr, s.pos, s.exp, c)
    wp = pts.shape[-1] // 2
    r = np.zeros((s.n_vars, 1, 4))
    r[:, 0, 0] = [abs(complex(pts[v, q, 0], pts[v, q, wp])) for v in range(s.n_vars)]
    return ms, r


def check_exact_moduli_route(fn, seed=11):
    """Scales equal the exact oracle's f and J of the moduli system."""
    s = _system(seed)
    pts = synth.points(seed + 1, s.n_vars, 3, modulus_octaves=(-2, 2))
    for q in range(3):
        Sf, SJ = fn(s, pts, q)
        ms, r = _moduli_system(s, pts, q)
        f, J = E.evaluate_point(ms, r, 0)
        for p in range(s.n_polys):
            want = E.cx_abs(f[p])
            if not math.isclose(Sf[p], want, rel_tol=1e-12, abs_tol=0.0):
                return False
            for i in range(s.n_vars):
                want = E.cx_abs(J[p].get(i, E.ZERO))
                if not math.isclose(SJ[p].get(i, 0.0), want, rel_tol=1e-12, abs_tol=0.0):
                    return False
    return True


def check_gradient_of_sf(fn, seed=12):
    """S_J[p][i] is the derivative of S_f[p] with respect to |x_i|."""
    s = _system(seed)
    pts = synth.points(seed + 1, s.n_vars, 1, modulus_octaves=(-1, 1))
    Sf, SJ = fn(s, pts, 0)
    h = 1e-5
    for i in range(s.n_vars):
        r = abs(complex(pts[i, 0, 0], pts[i, 0, 2]))
        up, dn = pts.copy(), pts.copy()
        up[i, 0] *= 1.0 + h
        dn[i, 0] *= 1.0 - h
        fu, _ = fn(s, up, 0)
        fd, _ = fn(s, dn, 0)
        for p in range(s.n_polys):
            g = (fu[p] - fd[p]) / (2 * h * r)
            scale = max(abs(SJ[p].get(i, 0.0)), Sf[p] / r, 1e-300)
            if abs(g - SJ[p].get(i, 0.0)) > 1e-7 * scale:
                return False
    return True


def check_euler_on_homogeneous(fn, seed=13):
    """sum_i |x_i| S_J[p][i] = d S_f[p] when every monomial has degree d."""
    s = synth.regular_system(seed, 10, 12, 4, 5, n_polys=3, coef_modulus=(-4, 4), homogeneous_degree=9)
    pts = synth.points(seed + 1, 10, 2, modulus_octaves=(-1, 1))
    for q in range(2):
        Sf, SJ = fn(s, pts, q)
        for p in range(s.n_polys):
            lhs = sum(abs(complex(pts[i, q, 0], pts[i, q, 2])) * SJ[p].get(i, 0.0) for i in range(s.n_vars))
            if not math.isclose(lhs, 9 * Sf[p], rel_tol=1e-12):
                return False
    return True


def check_speelpenning_powers_of_two(fn, seed=14):
    """x_1 ... x_k with |x_i| = 2^e_i (any phase) and |c| = 2^-3:
    S_f = 2^(sum e - 3) and S_J[i] = 2^(sum e - e_i - 3), exactly; and
    x_1^2 x_2^3 with |x| = (2, 4): S_J = (2*2*64, 3*4*16) / 8."""
    k = 5
    e = [1, -2, 3, 0, 2]
    s = synth.from_monomials(k, [[(list(range(k)), [1] * k)]], [[0.125 * 0.6, 0.0, 0.125 * 0.8, 0.0]])
    rng = np.random.Generator(np.random.PCG64(seed))
    pts = np.zeros((k, 1, 4))
    for i in range(k):
        # a Pythagorean phase (3/5, 4/5 and its quarter turns) keeps |x_i| exact
        re, im = [(0.6, 0.8), (-0.8, 0.6), (-0.6, -0.8), (0.8, -0.6)][int(rng.integers(0, 4))]
        pts[i, 0, 0], pts[i, 0, 2] = math.ldexp(re, e[i]), math.ldexp(im, e[i])
    Sf, SJ = fn(s, pts, 0)
    if Sf[0] != math.ldexp(1.0, sum(e) - 3):
        return False
    if any(SJ[0].get(i, 0.0) != math.ldexp(1.0, sum(e) - e[i] - 3) for i in range(k)):
        return False
    s2 = synth.from_monomials(2, [[([0, 1], [2, 3])]], [[1.0, 0.0, 0.0, 0.0]])
    p2 = np.zeros((2, 1, 4))
    p2[0, 0, 2], p2[1, 0, 0] = 2.0, -4.0
    Sf, SJ = fn(s2, p2, 0)
    return Sf[0] == 4.0 * 64.0 and SJ[0].get(0, 0.0) == 2 * 2 * 64.0 and SJ[0].get(1, 0.0) == 3 * 4 * 16.0


def check_absent_variables_zero(fn, seed=15):
    """S_J[p][i] is 0 exactly when x_i occurs in no monomial of p, and > 0 otherwise."""
    s = _system(seed, n=9, m=3, kmax=3)
    pts = synth.points(seed + 1, s.n_vars, 1)
    _, SJ = fn(s, pts, 0)
    for p in range(s.n_polys):
        occurs = set()
        for t in range(int(s.poly_ptr[p]), int(s.poly_ptr[p + 1])):
            occurs.update(s.monomial(t)[0])
        for i in range(s.n_vars):
            if (SJ[p].get(i, 0.0) > 0.0) != (i in occurs):
                return False
    return True


PINS = [check_exact_moduli_route, check_gradient_of_sf, check_euler_on_homogeneous,
        check_speelpenning_powers_of_two, check_absent_variables_zero]


@pytest.mark.parametrize("vectorised", [False, True], ids=["scales_point", "vectorised"])
@pytest.mark.parametrize("pin", PINS, ids=lambda c: c.__name__)
def test_scales_pin(pin, vectorised):
    assert pin(_point_fn(vectorised))


@pytest.mark.parametrize("cfg", [1, 2, 3])
def test_both_implementations_agree_on_workloads(cfg):
    s, pts = synth.config(cfg, n_points=3)
    Sf, SJ = vec_scales(s, pts)
    for q in range(pts.shape[1]):
        polys = [0, s.n_polys - 1]
        f, J = E.scales_point(s, pts, q, polys=polys)
        for p in polys:
            assert math.isclose(Sf[p, q], f[p], rel_tol=1e-12)
            for i in range(s.n_vars):
                assert math.isclose(SJ[p, i, q], J[p].get(i, 0.0), rel_tol=1e-12, abs_tol=0.0)


# ----------------------------------------------------------------------------
# planted mistakes: copies of the two implementations with one mistake each
# ----------------------------------------------------------------------------

def _mut_point(kind):
    """scales_point with a planted mistake."""
    def fn(system, pts, q):
        wp = pts.shape[-1] // 2
        wc = system.coef.shape[-1] // 2
        ax = {}
        for v in range(system.n_vars):
            ax[v] = abs(pts[v, q, 0]) if kind == "point_real_part" else math.hypot(pts[v, q, 0], pts[v, q, wp])
        Sf, SJ = {}, {}
        for p in range(system.n_polys):
            sf, sj = 0.0, {}
            for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
                pos, exp = system.monomial(t)
                ac = abs(system.coef[t, 0]) if kind == "coef_real_part" else math.hypot(system.coef[t, 0],
                                                                                        system.coef[t, wc])
                term = ac
                for v, a in zip(pos, exp):
                    term *= ax[v] ** a
                sf += term
                for i, ai in zip(pos, exp):
                    d = ac if kind == "dropped_exponent_factor" else ac * ai
                    for v, a in zip(pos, exp):
                        d *= ax[v] ** (a if (v != i or kind == "exponent_not_lowered") else a - 1)
                    sj[i] = sj.get(i, 0.0) + d
            Sf[p], SJ[p] = sf, sj
        return Sf, SJ

    return fn


def _mut_vectorised(kind):
    """tests/_util.scales at one point, with a planted mistake."""
    def fn(system, pts, q):
        n, N, M = system.n_vars, system.n_polys, system.n_monos
        k = np.diff(system.mono_ptr).astype(np.int64)
        kmax = max(int(k.max()) if k.size else 0, 1)
        poly_of = np.repeat(np.arange(N), np.diff(system.poly_ptr))
        w = system.coef.shape[1] // 2
        ac = np.abs(system.coef[:, 0]) if kind == "coef_real_part" else np.hypot(system.coef[:, 0],
                                                                                 system.coef[:, w])
        rows = np.repeat(np.arange(M), k)
        cols = np.arange(system.pos.size) - np.repeat(system.mono_ptr[:-1], k)
        ax = (np.abs(pts[:, q, 0]) if kind == "point_real_part"
              else np.hypot(pts[:, q, 0], pts[:, q, pts.shape[-1] // 2]))
        W = np.ones((M, kmax))
        Wd = np.ones((M, kmax))
        W[rows, cols] = ax[system.pos] ** system.exp
        fac = 1 if kind == "dropped_exponent_factor" else system.exp
        low = 0 if kind == "exponent_not_lowered" else 1
        Wd[rows, cols] = fac * ax[system.pos] ** (system.exp - low)
        pre = np.cumprod(np.concatenate([np.ones((M, 1)), W[:, :-1]], axis=1), axis=1)
        suf = np.cumprod(np.concatenate([np.ones((M, 1)), W[:, :0:-1]], axis=1), axis=1)[:, ::-1]
        Sf = np.zeros(N)
        SJ = np.zeros((N, n))
        np.add.at(Sf, poly_of, ac * pre[:, -1] * W[:, -1])
        np.add.at(SJ, (poly_of[rows], system.pos), ac[rows] * Wd[rows, cols] * pre[rows, cols] * suf[rows, cols])
        return ({p: float(Sf[p]) for p in range(N)},
                {p: {i: float(SJ[p, i]) for i in range(n) if SJ[p, i] != 0.0} for p in range(N)})

    return fn


MISTAKES = ["dropped_exponent_factor", "exponent_not_lowered", "coef_real_part", "point_real_part"]


@pytest.mark.parametrize("impl", ["scales_point", "vectorised"])
@pytest.mark.parametrize("kind", MISTAKES)
def test_planted_scale_mistake_is_caught(kind, impl):
    fn = _mut_point(kind) if impl == "scales_point" else _mut_vectorised(kind)
    results = []
    for pin in PINS:
        try:
            results.append(pin(fn))
        except Exception:
            results.append(False)
    assert not all(results), f"{kind} in {impl} survived every pin"


@pytest.mark.parametrize("impl", ["scales_point", "vectorised"])
def test_unmutated_copies_pass(impl):
    """The mutation scaffolding itself, with no mistake planted, passes every
    pin (so a caught mistake is the mistake, not the copy)."""
    fn = _mut_point("none") if impl == "scales_point" else _mut_vectorised("none")
    assert all(pin(fn) for pin in PINS)
