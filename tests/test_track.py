"""Path tracking on the GPU (polyeval_start_points, polyeval_track,
polyeval_track_adaptive) against the tracking oracle and known solution sets.

End points are compared as sets (the paths may meet the solutions in any
order): every expected solution must have its own GPU end point within the
tolerance.  Double-double end points are also checked by their exact
residual |F(x*)| / S_F(x*) from the exact oracle.
"""
import itertools

import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import track as T

from _util import pe_precision

pytestmark = pytest.mark.gpu

TRACK_PRECS = ["dd", "ddint", "f64"]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1201_0499_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(0)


def system_for(s, prec):
    return s.as_fp64() if prec == "f64" else s


def run_track(s, prec, prm=None):
    """(end points [B, n] complex, raw end points [n, B, c], status [B], handle)."""
    import torch

    import paper_1201_0499_gb300 as pkg

    B = int(np.prod(T.degrees(s)))
    ev = pkg.PolyEval(system_for(s, prec), pe_precision(prec), max_points=B)
    assert ev.bezout()[0] == B
    x = ev.start_points(B)
    status, t, it = ev.track(x, prm)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK and it >= 1
    raw = x.cpu().numpy()
    w = raw.shape[-1] // 2
    z = (raw[..., 0] + 1j * raw[..., w]).T
    return z, raw, status.cpu().numpy(), t.cpu().numpy(), ev


def match(found, want, tol):
    found = [np.asarray(f) for f in found]
    used = set()
    for w in want:
        d = [(np.max(np.abs(f - np.asarray(w))), i) for i, f in enumerate(found) if i not in used]
        best, i = min(d)
        if best > tol:
            return False
        used.add(i)
    return True


def exact_residual(s, raw):
    """max over paths and polynomials of |F(x*)| / S_F(x*), exactly."""
    worst = 0.0
    for q in range(raw.shape[1]):
        f, _ = E.evaluate_point(s, raw, q)
        Sf, _ = E.scales_point(s, raw, q)
        for p in range(s.n_polys):
            worst = max(worst, E.cx_abs(f[p]) / Sf[p])
    return worst


def univariate(seed, deg):
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal(deg + 1) + 1j * rng.standard_normal(deg + 1)
    mons = [([0], [k]) if k else ([], []) for k in range(deg + 1)]
    return synth.from_monomials(1, [mons], [[z.real, 0, z.imag, 0] for z in c]), c


@pytest.mark.parametrize("prec", TRACK_PRECS)
def test_track_univariate_matches_numpy_roots(prec):
    s, c = univariate(611, 7)
    z, raw, st, t, _ = run_track(s, prec)
    assert np.all(st == 1) and np.all(t == 1.0)
    assert match(list(z), [[r] for r in np.roots(c[::-1])], 1e-9)


@pytest.mark.parametrize("prec", TRACK_PRECS)
def test_track_decoupled_product_set(prec):
    r0 = [0.5 + 0.25j, -1.0 + 0.5j, 0.2 - 1.1j]
    r1 = [1.5j, -0.75]
    polys, coef = [], []
    for v, roots in ((0, r0), (1, r1)):
        c = np.array([1.0 + 0j])
        for r in roots:
            c = np.convolve(c, [1.0, -r])
        mons = []
        for k, a in enumerate(c):
            e = len(roots) - k
            mons.append(([v], [e]) if e else ([], []))
            coef.append([a.real, 0, a.imag, 0])
        polys.append(mons)
    s = synth.from_monomials(2, polys, coef)
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == 6 and np.all(st == 1)
    assert match(list(z), list(itertools.product(r0, r1)), 1e-9)


@pytest.mark.parametrize("prec", TRACK_PRECS)
@pytest.mark.parametrize("case", [(612, 3, [2, 2, 2]), (613, 4, [2, 3, 1, 2])], ids=["n3_deg222", "n4_deg2312"])
def test_track_generic_matches_oracle(prec, case):
    seed, n, degs = case
    s = synth.dense_system(seed, n, degs)
    ref = T.solve_system(s.as_fp64() if prec == "f64" else s)
    assert all(stv == T.SUCCESS for _, stv in ref)
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == len(ref) and np.all(st == 1)
    assert match(list(z), [x for x, _ in ref], 1e-8)
    if prec != "f64":
        assert exact_residual(s, raw) <= 1e-24


@pytest.mark.parametrize("prec", TRACK_PRECS)
def test_track_nine_variables_sixteen_lane_segments(prec):
    """n = 9 (16 lanes per path, two paths per warp) against the oracle."""
    s = synth.dense_system(621, 9, [2, 2, 2, 1, 1, 1, 1, 1, 1])
    ref = T.solve_system(s.as_fp64() if prec == "f64" else s)
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == 8 and np.all(st == 1)
    assert match(list(z), [x for x, _ in ref], 1e-8)
    if prec != "f64":
        assert exact_residual(s, raw) <= 1e-24


def test_track_start_points_on_device():
    import torch

    import paper_1201_0499_gb300 as pkg

    s = synth.dense_system(614, 3, [2, 3, 2])
    for prec in ("dd", "f64"):
        ev = pkg.PolyEval(system_for(s, prec), pe_precision(prec), max_points=12)
        assert ev.bezout() == (12.0, [2, 3, 2])
        x = ev.start_points(7, first=5)
        torch.cuda.synchronize()
        raw = x.cpu().numpy()
        w = raw.shape[-1] // 2
        want = T.start_points([2, 3, 2])[5:12]
        for j in range(7):
            for i in range(3):
                assert abs(complex(raw[i, j, 0], raw[i, j, w]) - want[j][i]) < 1e-15
                if w == 2:
                    assert raw[i, j, 1] == 0.0 and raw[i, j, 3] == 0.0


def test_track_dense_six_quadrics():
    """64 paths of a generic system of six quadrics in six variables, in
    double-double: all succeed at distinct end points with tiny residuals."""
    s = synth.dense_system(615, 6, [2] * 6)
    z, raw, st, _, _ = run_track(s, "dd")
    assert len(st) == 64 and np.all(st == 1)
    d = np.abs(z[:, None, :] - z[None, :, :]).max(axis=2) + np.eye(64)
    assert d.min() > 1e-6
    assert exact_residual(s, raw) <= 1e-24


@pytest.mark.parametrize("hi", ["dd", "ddint"])
def test_track_adaptive_precision(hi):
    import torch

    import paper_1201_0499_gb300 as pkg

    s = synth.dense_system(616, 4, [2, 2, 3, 1])
    B = 12
    lo = pkg.PolyEval(s.as_fp64(), pkg.PE_F64, max_points=B)
    hh = pkg.PolyEval(s, pe_precision(hi), max_points=B)
    prm_lo = pkg.polyeval_track_defaults(pkg.PE_F64)
    prm_hi = pkg.polyeval_track_defaults(pe_precision(hi))
    ref = T.solve_system(s.as_fp64())
    for force in (False, True):
        x = hh.start_points(B)
        status = torch.empty(B, dtype=torch.int32, device="cuda")
        p_lo = prm_lo
        if force:  # a double-precision end tolerance no double can meet: every path escalates
            p_lo = pkg.polyeval_track_defaults(pkg.PE_F64)
            p_lo.end_tol = 1e-300
            p_lo.max_end = 2
        esc = pkg.polyeval_track_adaptive(lo.handle, hh.handle, p_lo, prm_hi, x, B, status)
        torch.cuda.synchronize()
        st = status.cpu().numpy()
        raw = x.cpu().numpy()
        assert np.all(st == 1)
        assert esc == B if force else 0 <= esc < B
        z = (raw[..., 0] + 1j * raw[..., 2]).T
        assert match(list(z), [xx for xx, _ in ref], 1e-8)
        assert exact_residual(s, raw) <= 1e-24


@pytest.mark.parametrize("mixed", [0, 1])
def test_track_double_double_linear_solves(mixed):
    """Double-double tracking with the linear systems in double-double
    (mixed = 0) or in double with double-double residuals (mixed = 1): the
    same solutions, at double-double accuracy either way."""
    import paper_1201_0499_gb300 as pkg

    s = synth.dense_system(618, 3, [2, 3, 2])
    prm = pkg.polyeval_track_defaults(pkg.PE_DD)
    prm.mixed = mixed
    z, raw, st, _, _ = run_track(s, "dd", prm)
    assert np.all(st == 1)
    assert match(list(z), [x for x, _ in T.solve_system(s)], 1e-8)
    assert exact_residual(s, raw) <= 1e-24


@pytest.mark.parametrize("mixed", [0, 1])
def test_track_large_system_two_paths(mixed):
    """n = 60: 59 dense linear equations and one quadric (2 paths).  The
    60 x 60 double-double system is too large for shared memory (solved in
    place in global memory); in double it is staged."""
    import paper_1201_0499_gb300 as pkg

    n = 60
    rng = np.random.Generator(np.random.PCG64(619))
    polys = [[([j], [1]) for j in range(n)] + [([], [])] for _ in range(n - 1)]
    polys.append([([0], [2]), ([1, 2], [1, 1]), ([3], [1]), ([], [])])
    M = sum(len(p) for p in polys)
    s = synth.from_monomials(n, polys, synth.random_cdd(rng, M))
    prm = pkg.polyeval_track_defaults(pkg.PE_DD)
    prm.mixed = mixed
    z, raw, st, _, _ = run_track(s, "dd", prm)
    assert len(st) == 2 and np.all(st == 1)
    assert np.max(np.abs(z[0] - z[1])) > 1e-6
    assert exact_residual(s, raw) <= 1e-24


@pytest.mark.parametrize("prec", ["f64", "dd"])
def test_track_large_batch(prec):
    """4096 paths (twelve quadrics, 16-lane segments, two paths per warp).
    Every path succeeds at a distinct end point; sampled end points have tiny
    exact residuals."""
    s = synth.dense_system(620, 12, [2] * 12)
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == 4096 and np.all(st == 1)
    keys = np.round(np.concatenate([z.real, z.imag], axis=1), 6)
    assert len(np.unique(keys, axis=0)) == 4096  # distinct end points
    sample = raw[:, ::97]
    tol = 1e-24 if prec == "dd" else 1e-12
    assert exact_residual(system_for(s, prec), np.ascontiguousarray(sample)) <= tol


@pytest.mark.parametrize("prec", ["f64", "dd"])
def test_track_half_the_paths_diverge(prec):
    """256 paths, 128 finite solutions: six decoupled quadrics with known
    roots and x6^2 = 1, x6 x7 = 2 (two finite solutions, the other two paths of
    that block go to infinity).  Half the paths end early, so the batch is
    compacted while the rest run; the successes must be exactly the 128
    solutions and the others must not succeed."""
    rng = np.random.Generator(np.random.PCG64(622))
    roots = [(complex(*rng.standard_normal(2)), complex(*rng.standard_normal(2))) for _ in range(6)]
    polys, coef = [], []
    for v, (r1, r2) in enumerate(roots):
        c = np.convolve([1.0, -r1], [1.0, -r2])
        polys.append([([v], [2]), ([v], [1]), ([], [])])
        coef += [[c[0].real, 0, c[0].imag, 0], [c[1].real, 0, c[1].imag, 0], [c[2].real, 0, c[2].imag, 0]]
    polys.append([([6], [2]), ([], [])])
    coef += [[1, 0, 0, 0], [-1, 0, 0, 0]]
    polys.append([([6, 7], [1, 1]), ([], [])])
    coef += [[1, 0, 0, 0], [-2, 0, 0, 0]]
    s = synth.from_monomials(8, polys, coef)
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == 256 and int(np.sum(st == 1)) == 128 and np.all(st != 0)
    want = [list(r) + [x6, 2 / x6] for r in itertools.product(*roots) for x6 in (1.0, -1.0)]
    assert match([z[i] for i in np.flatnonzero(st == 1)], want, 1e-9)


@pytest.mark.parametrize("prec", ["f64", "dd"])
def test_track_paths_that_overflow_end_diverged(prec):
    """x0^2 = 1/4 and 1e307 x1^2 - 1e307 x1^2 + x1 - 1/2 = 0: the two
    x1^2 terms cancel exactly while they are finite, so F is x1 - 1/2 there,
    but the total degree is 2 and one path of each x0 root goes to infinity.
    Past |x1| = 4.3 both terms overflow and F(x) = inf - inf = NaN.  A NaN in
    one coordinate of a step must not be dropped by the step-size test (a max
    that skips NaN would accept the step on the finite coordinate and carry
    the NaN on to a "success"): the two finite solutions succeed with finite
    coordinates, the two other paths end diverged."""
    s = synth.from_monomials(2, [[([0], [2]), ([], [])], [([1], [2]), ([1], [2]), ([1], [1]), ([], [])]],
                             [[1, 0, 0, 0], [-0.25, 0, 0, 0], [1e307, 0, 0, 0], [-1e307, 0, 0, 0],
                              [1, 0, 0, 0], [-0.5, 0, 0, 0]])
    z, raw, st, _, _ = run_track(s, prec)
    ok = st == 1
    assert int(np.sum(ok)) == 2 and np.all(np.isfinite(z[ok])), (st, z)
    assert np.all(st[~ok] == 3), st
    assert match([z[i] for i in np.flatnonzero(ok)], [[0.5, 0.5], [-0.5, 0.5]], 1e-9)


@pytest.mark.parametrize("prec", ["f64", "dd"])
def test_track_double_root_is_not_reported_as_converged(prec):
    """(x - 1)^2 = 0, y^2 = 2: every path ends at a double root in x, where
    Newton's method converges only linearly, so no path may report success;
    the paths end either with a failed step size or with a non-converged end
    point, and then near x = 1 with y^2 = 2."""
    s = synth.from_monomials(2, [[([0], [2]), ([0], [1]), ([], [])], [([1], [2]), ([], [])]],
                             [[1, 0, 0, 0], [-2, 0, 0, 0], [1, 0, 0, 0], [1, 0, 0, 0], [-2, 0, 0, 0]])
    z, raw, st, _, _ = run_track(s, prec)
    assert len(st) == 4 and np.all((st == 2) | (st == 4)), st
    for q in np.flatnonzero(st == 4):
        assert abs(z[q, 0] - 1) < 1e-3 and abs(z[q, 1] ** 2 - 2) < 1e-6


def test_track_no_finite_solutions():
    s = synth.from_monomials(2, [[([0, 1], [1, 1]), ([], [])], [([0, 1], [1, 1]), ([], [])]],
                             [[1, 0, 0, 0], [-1, 0, 0, 0], [1, 0, 0, 0], [-2, 0, 0, 0]])
    _, _, st, _, _ = run_track(s, "f64")
    assert np.all(st != 1) and np.all(st != 0)


def test_track_rejections():
    import torch

    import paper_1201_0499_gb300 as pkg

    rect = synth.from_monomials(3, [[([0], [1])], [([1], [2])]], [[1, 0, 0, 0], [1, 0, 0, 0]])
    ev = pkg.PolyEval(rect, pkg.PE_DD, max_points=4)
    with pytest.raises(pkg.PolyEvalError) as e:
        ev.start_points(4)
    assert e.value.code == pkg.PE_EINVAL
    const = synth.from_monomials(2, [[([0], [1])], [([], [])]], [[1, 0, 0, 0], [1, 0, 0, 0]])
    ev = pkg.PolyEval(const, pkg.PE_DD, max_points=4)
    with pytest.raises(pkg.PolyEvalError) as e:
        ev.track(torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda"))
    assert e.value.code == pkg.PE_EINVAL
    s = synth.dense_system(617, 2, [2, 2])
    evq = pkg.PolyEval(s, pkg.PE_QD_INT, max_points=4)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_start_points(evq.handle, 0, 4, torch.zeros((2, 4, 8), dtype=torch.float64, device="cuda"))
    assert e.value.code == pkg.PE_EINVAL
    ev = pkg.PolyEval(s, pkg.PE_DD, max_points=2)
    with pytest.raises(pkg.PolyEvalError) as e:
        ev.track(torch.zeros((2, 4, 4), dtype=torch.float64, device="cuda"))
    assert e.value.code == pkg.PE_ERANGE
