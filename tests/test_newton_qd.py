"""Newton's method on a quad-double handle (PE_QD_INT): f and J evaluated in
quad-double, the correction solved in double-double from their leading parts,
x + dx rounded to quad-double (the corrector of Section 1 at the precision of
the QD library).

* One step against the exact Newton step of the oracle: the backward error of
  dx measured with the exact f and J, the update x1 = x0 + dx to quad-double
  accuracy, x1 normalised, the lower parts of dx and of the factors zero.
  n = 5 and 12 stage the solve in shared memory, n = 24 in device scratch.
* The benchmark system (n = 32, m = 64, k = 9) shifted to have a quad-double
  root x*: points near x* converge to it at quad-double accuracy, far past
  what a double-double Newton step can reach.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E
from oracle import newton as N

from _util import cabs, fr_parts, square_system, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)


def ulp(x):
    _, e = np.frexp(np.abs(x))
    return np.ldexp(1.0, (e - 53).astype(np.int32))


def assert_normalised(arr):
    for c in (0, 4):
        parts = arr.reshape(-1, 8)[:, c:c + 4]
        for i in range(3):
            hi, lo = parts[:, i], parts[:, i + 1]
            assert np.all(np.abs(lo) <= ulp(hi) / 2)
            assert np.all((hi != 0) | (lo == 0))


def newton_qd(system, pts, steps=1):
    import torch

    import paper_1201_0499_gb300 as pkg

    ev = pkg.PolyEval(system, pkg.PE_QD_INT, max_points=pts.shape[1])
    x = to_device(pts)
    norms = []
    for _ in range(steps):
        dx, lu, nm = ev.newton(x)
        torch.cuda.synchronize()
        norms.append(nm.cpu().numpy())
    assert ev.status() == pkg.PE_OK
    out = x.cpu().numpy(), dx.cpu().numpy(), lu.cpu().numpy(), norms
    ev.close()
    return out


@pytest.mark.parametrize("n", [5, 12, 24])
def test_qd_newton_step_against_exact(n):
    P = 19
    rng = np.random.Generator(np.random.PCG64(610 + n))
    s = square_system(611, n, m=6, kmax=3, emax=3).to_qd(612)
    pts = synth.widen_qd(rng, synth.points(613, n, P))
    x1, dx, lu, norms = newton_qd(s, pts)
    assert np.all(dx[..., [2, 3, 6, 7]] == 0.0) and np.all(lu[..., [2, 3, 6, 7]] == 0.0)
    assert_normalised(x1)
    for q in (0, 7, P - 1):
        f, J = N.f_and_J(s, pts, q)
        g = [fr_parts(dx[i, q]) for i in range(n)]
        # dx solves the leading parts of J and f in double-double: its
        # backward error against the exact J and f is that of the solve
        res = 0.0
        for i in range(n):
            acc = f[i]
            for j in range(n):
                acc = N.c_add(acc, N.c_mul(J[i][j], g[j]))
            res = max(res, cabs(acc))
        Jn = max(sum(cabs(J[i][j]) for j in range(n)) for i in range(n))
        fn = max(cabs(fi) for fi in f)
        gn = max(cabs(gi) for gi in g)
        assert res / (Jn * gn + fn) <= 1e-28, q
        # x1 = x0 + dx, rounded to quad-double
        for i in range(n):
            want = N.c_add(fr_parts(pts[i, q]), g[i])
            assert cabs(N.c_sub(fr_parts(x1[i, q]), want)) <= 1e-62 * cabs(want), (q, i)
        assert norms[0][q, 0] == pytest.approx(fn, rel=1e-12)
        assert norms[0][q, 1] == pytest.approx(gn, rel=1e-12)


def shifted_qd_system(system, root):
    """system - system(x*) with quad-double coefficients: a constant term per
    polynomial equal to -f_p(x*) rounded to quad-double, so that the
    quad-double point x* is a root up to that rounding."""
    polys, coef = [], []
    for p in range(system.n_polys):
        mons = []
        for t in range(int(system.poly_ptr[p]), int(system.poly_ptr[p + 1])):
            mons.append(system.monomial(t))
            coef.append(system.coef[t])
        mons.append(([], []))
        coef.append(np.zeros(4))
        polys.append(mons)
    s = synth.from_monomials(system.n_vars, polys, np.asarray(coef)).to_qd(701)
    f, _J = E.evaluate_point(s, root, 0)
    for p in range(s.n_polys):
        t = next(t for t in range(int(s.poly_ptr[p]), int(s.poly_ptr[p + 1]))
                 if s.mono_ptr[t + 1] == s.mono_ptr[t])
        s.coef[t] = E.cx_to_qd(E.cx_sub(E.ZERO, f[p]))
    return s


def test_qd_newton_converges_to_quad_double_accuracy():
    g, _ = synth.config(2, n_points=1)
    n, P = g.n_vars, 256
    rng = np.random.Generator(np.random.PCG64(702))
    root = synth.widen_qd(rng, synth.points(703, n, 1))
    s = shifted_qd_system(g, root)
    start = np.repeat(root, P, axis=1)
    start[..., 0] *= 1.0 + 1e-7 * rng.standard_normal((n, P))
    start[..., 4] *= 1.0 + 1e-7 * rng.standard_normal((n, P))
    x, _dx, _lu, norms = newton_qd(s, start, steps=6)
    steps = [float(nm[:, 1].max()) for nm in norms]
    assert steps[0] < 1e-5 and steps[1] < 1e-9 and steps[2] < 1e-20, steps
    assert steps[-1] < 1e-58, steps
    err = 0.0
    for q in range(0, P, 37):
        for i in range(n):
            err = max(err, cabs(N.c_sub(fr_parts(x[i, q]), fr_parts(root[i, 0]))))
    assert err < 1e-58, err
    assert_normalised(x)


def test_qd_newton_singular_point_and_empty_batch():
    """A point where the Jacobian is exactly zero (x = 0 on x_i^2 + c_i) is
    left unchanged with dx = 0 and a NaN step norm; its neighbour in the
    batch still takes its step.  An empty batch is a no-op."""
    import torch

    import paper_1201_0499_gb300 as pkg

    rng = np.random.Generator(np.random.PCG64(720))
    n = 3
    polys = [[([i], [2]), ([], [])] for i in range(n)]
    s = synth.from_monomials(n, polys, synth.random_cdd(rng, 2 * n)).to_qd(721)
    pts = synth.widen_qd(rng, synth.points(722, n, 2))
    pts[:, 0, :] = 0.0
    x1, dx, _lu, norms = newton_qd(s, pts)
    assert np.all(x1[:, 0] == 0.0) and np.all(dx[:, 0] == 0.0)
    assert np.isnan(norms[0][0, 1]) and norms[0][1, 1] > 0.0
    f, J, _dx, _x1 = N.newton_step(s, pts, 1)
    for i in range(n):
        want = N.c_add(fr_parts(pts[i, 1]), N.c_div(N.c_sub(N.ZERO, f[i]), J[i][i]))
        assert cabs(N.c_sub(fr_parts(x1[i, 1]), want)) <= 1e-28 * cabs(want)
    ev = pkg.PolyEval(s, pkg.PE_QD_INT, max_points=4)
    x = torch.empty((n, 0, 8), dtype=torch.float64, device="cuda")
    ev.newton(x)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
