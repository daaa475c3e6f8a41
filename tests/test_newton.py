"""Newton's method on the GPU (polyeval_newton): one step x <- x + dx with
J(x) dx = -f(x), the corrector the paper's evaluation serves (Section 1).

* Small square systems: the GPU step against the oracle's exact f and J:
  the normwise backward error |J dx + f| / (|J| |dx| + |f|) of the GPU dx,
  measured with the exact J and f, and the update x1 = x0 + dx.
* The benchmark system (n = 32, m = 64, k = 9) shifted to have a root x*:
  1024 points near x* converge quadratically to it.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import newton as N

from _util import PRECS, cabs, fr_parts as fr_dd, pe_precision, square_system, to_device, widen

pytestmark = pytest.mark.gpu

BACKWARD_TOL = {"dd": 1e-28, "ddint": 1e-28, "f64": 1e-14}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def run_newton(system, pts, prec):
    import torch

    import paper_1201_0499_gb300 as pkg

    dd = prec != "f64"
    ev = pkg.PolyEval(system if dd else system.as_fp64(), pe_precision(prec), max_points=pts.shape[1])
    x = to_device(pts, dd)
    dx, _lu, norms = ev.newton(x)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    x1, dx = x.cpu().numpy(), dx.cpu().numpy()
    if not dd:
        x1, dx = widen(x1), widen(dx)
    return x1, dx, norms.cpu().numpy()


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("n", [5, 12])
def test_newton_step_against_exact(prec, n):
    P = 21
    s = square_system(201, n, m=6, kmax=3, emax=3)
    pts = synth.points(202, n, P)
    if prec == "f64":
        s, pts = s.as_fp64(), pts.copy()
        pts[..., 1] = 0.0
        pts[..., 3] = 0.0
    x1, dx, norms = run_newton(s, pts, prec)
    for q in range(P):
        f, J = N.f_and_J(s, pts, q)
        g = [fr_dd(dx[i, q]) for i in range(n)]
        # backward error of the GPU step against the exact f and J
        res = 0.0
        for i in range(n):
            acc = f[i]
            for j in range(n):
                acc = N.c_add(acc, N.c_mul(J[i][j], g[j]))
            res = max(res, cabs(acc))
        Jn = max(sum(cabs(J[i][j]) for j in range(n)) for i in range(n))
        fn = max(cabs(fi) for fi in f)
        gn = max(cabs(gi) for gi in g)
        eta = res / (Jn * gn + fn)
        assert eta <= BACKWARD_TOL[prec], (q, eta)
        # the update: x1 = x0 + dx (renormalised)
        for i in range(n):
            want = N.c_add(fr_dd(pts[i, q]), g[i])
            assert cabs(N.c_sub(fr_dd(x1[i, q]), want)) <= 1e-30 * cabs(want) + (1e-15 * cabs(want) if prec == "f64" else 0)
        # the reported norms
        assert norms[q, 0] == pytest.approx(max(cabs(fi) for fi in f), rel=1e-12)
        assert norms[q, 1] == pytest.approx(gn, rel=1e-12)


def shifted_system(system, root_pts):
    """system - system(x*): the constant term of each polynomial is lowered by
    f_p(x*) (exact value rounded to double-double), so x* is a root up to that
    rounding."""
    f, _J = E.evaluate_point(system, root_pts, 0)
    polys = []
    coef = []
    for p in range(system.n_polys):
        mons = []
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            mons.append(system.monomial(t))
            coef.append(system.coef[t])
        mons.append(([], []))
        c = E.cx_to_dd(E.cx_sub(E.ZERO, f[p]))
        coef.append(list(c))
        polys.append(mons)
    return synth.from_monomials(system.n_vars, polys, np.asarray(coef))


@pytest.mark.parametrize("prec", ["dd", "ddint", "f64"])
def test_newton_converges_on_the_benchmark_system(prec):
    import torch

    import paper_1201_0499_gb300 as pkg

    g, _ = synth.config(2, n_points=1)
    n, P = g.n_vars, 1024
    root = synth.points(301, n, 1)
    s = shifted_system(g, root)
    rng = np.random.Generator(np.random.PCG64(302))
    start = np.repeat(root, P, axis=1)
    start[..., 0] *= 1.0 + 1e-7 * rng.standard_normal((n, P))
    start[..., 2] *= 1.0 + 1e-7 * rng.standard_normal((n, P))
    start[..., 1] = 0.0
    start[..., 3] = 0.0
    dd = prec != "f64"
    ev = pkg.PolyEval(s if dd else s.as_fp64(), pe_precision(prec), max_points=P)
    x = to_device(start, dd)
    steps = []
    for _ in range(5):
        _dx, _lu, norms = ev.newton(x)
        torch.cuda.synchronize()
        steps.append(float(norms[:, 1].max()))
    assert ev.status() == pkg.PE_OK
    xf = x.cpu().numpy()
    if not dd:
        xf = widen(xf)
    # quadratic convergence: the step sizes fall to the precision's floor
    assert steps[0] < 1e-5 and steps[1] < 1e-9
    floor = 1e-26 if dd else 1e-12
    assert steps[-1] < floor, steps
    err = np.abs((xf[..., 0] - root[..., 0]) + (xf[..., 1] - root[..., 1])) + \
        np.abs((xf[..., 2] - root[..., 2]) + (xf[..., 3] - root[..., 3]))
    assert float(err.max()) < floor, float(err.max())


@pytest.mark.parametrize("prec", ["dd", "f64"])
def test_newton_large_batch_small_system(prec):
    """4096 points of an 8 x 8 system (8-lane segments, four points per
    warp).  The step is checked against the exact Newton step at sampled
    points."""
    n, P = 8, 4096
    s = square_system(205, n, m=5, kmax=3, emax=3)
    pts = synth.points(206, n, P)
    if prec == "f64":
        s, pts = s.as_fp64(), pts.copy()
        pts[..., 1] = 0.0
        pts[..., 3] = 0.0
    x1, dx, norms = run_newton(s, pts, prec)
    for q in (0, 1, 2047, 4095):
        f, J = N.f_and_J(s, pts, q)
        g = [fr_dd(dx[i, q]) for i in range(n)]
        res = 0.0
        for i in range(n):
            acc = f[i]
            for j in range(n):
                acc = N.c_add(acc, N.c_mul(J[i][j], g[j]))
            res = max(res, cabs(acc))
        Jn = max(sum(cabs(J[i][j]) for j in range(n)) for i in range(n))
        eta = res / (Jn * max(cabs(gi) for gi in g) + max(cabs(fi) for fi in f))
        assert eta <= BACKWARD_TOL[prec], (q, eta)
        assert norms[q, 1] == pytest.approx(max(cabs(gi) for gi in g), rel=1e-12)


def test_newton_rejects_non_square_and_batch():
    import torch

    import paper_1201_0499_gb300 as pkg

    s = square_system(203, 4, m=3, kmax=2, emax=2)
    rect = synth.from_monomials(4, [[([0], [1])]] * 3, synth.random_cdd(np.random.Generator(np.random.PCG64(1)), 3))
    ev = pkg.PolyEval(rect, pkg.PE_DD, max_points=4)
    x = to_device(synth.points(204, 4, 4))
    with pytest.raises(pkg.PolyEvalError) as e:
        ev.newton(x, out_J=torch.empty((3, 4, 4, 4), dtype=torch.float64, device="cuda"))
    assert e.value.code == pkg.PE_EINVAL
    many = pkg.PolyEvalMany([s], [4], pkg.PE_DD)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_newton(many.handle, x, 4, x, x)
    assert e.value.code == pkg.PE_EINVAL


@pytest.mark.parametrize("prec", ["dd", "ddint", "f64"])
def test_newton_step_on_the_n128_system(prec):
    """One Newton step on the n = 128, m = 1024, k = 32 system at 48 points
    (128 x 128 complex systems, solved in global memory by 32-lane segments):
    at four of the points the normwise backward error of the GPU dx, measured
    exactly against the C double-double oracle's f and J (themselves within
    1e-30 of exact), is within the precision's bound."""
    import oracle

    s, pts = synth.config(5, n_points=48)
    n = s.n_vars
    if prec == "f64":
        s, pts = s.as_fp64(), pts.copy()
        pts[..., 1] = 0.0
        pts[..., 3] = 0.0
    _x1, dx, norms = run_newton(s, pts, prec)
    sample = [0, 17, 40, 47]
    Fo, Jo = oracle.dd_eval(s, np.ascontiguousarray(pts[:, sample]), threads=0)
    for c, q in enumerate(sample):
        f = [fr_dd(Fo[i, c]) for i in range(n)]
        g = [fr_dd(dx[i, q]) for i in range(n)]
        res, Jn = 0.0, 0.0
        for i in range(n):
            row = [fr_dd(Jo[i, j, c]) for j in range(n)]
            acc = f[i]
            for j in range(n):
                acc = N.c_add(acc, N.c_mul(row[j], g[j]))
            res = max(res, cabs(acc))
            Jn = max(Jn, sum(cabs(v) for v in row))
        gn = max(cabs(gi) for gi in g)
        eta = res / (Jn * gn + max(cabs(fi) for fi in f))
        assert eta <= BACKWARD_TOL[prec], (q, eta)
        assert norms[q, 1] == pytest.approx(gn, rel=1e-12)
