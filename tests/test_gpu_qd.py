"""Parity of the quad-double path (PE_QD_INT) with the exact oracle.

Inputs are genuine quad-doubles: the double-double coefficients and points
of the other tests with two random lower parts each (``synth.widen_qd``), so
that an implementation reading only the leading two parts fails.  Tolerance:
normwise 1e-60 (``QD_TOL``); Gaussian-integer data whose results stay below
2**53 must come out exactly, as (value, +0, +0, +0) per component.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import QD_TOL, to_device

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1201_0499_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(0)


def run_qd(system, pts, max_points=None):
    """f [N, P, 8], J [N, n, P, 8] from the CUDA library."""
    import torch

    import paper_1201_0499_gb300 as pkg

    P = pts.shape[1]
    ev = pkg.PolyEval(system, pkg.PE_QD_INT, max_points=max(P, 1) if max_points is None else max_points)
    f, J = ev.eval(to_device(pts))
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    f, J = f.cpu().numpy(), J.cpu().numpy()
    ev.close()
    return f, J


def qd_data(seed, system, pts):
    """The system's coefficients and the points widened to quad-double."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return system.to_qd(seed + 1), synth.widen_qd(rng, pts)


def check_exact(system, pts, f, J, points_idx=None, polys=None, tol=QD_TOL):
    idx = range(pts.shape[1]) if points_idx is None else points_idx
    ef, ej = E.max_errors(system, pts, f, J, idx, polys=polys)
    assert ef <= tol and ej <= tol, (ef, ej)
    return ef, ej


def random_system(seed, n, N, m, kmin, kmax, emax, coef_mod=None):
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _p in range(N):
        mons = []
        for _t in range(m):
            k = int(rng.integers(kmin, kmax + 1))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, emax + 1, size=k).tolist()))
        polys.append(mons)
    mod = None
    if coef_mod is not None:
        mod = np.ldexp(1.0 + rng.random(N * m), rng.integers(coef_mod[0], coef_mod[1] + 1, size=N * m))
    return synth.from_monomials(n, polys, synth.random_cdd(rng, N * m, mod))


def ulp(x):
    _, e = np.frexp(np.abs(x))
    return np.ldexp(1.0, (e - 53).astype(np.int32))


def test_qd_several_tiles_ragged_tail():
    s = random_system(401, n=20, N=12, m=10, kmin=1, kmax=7, emax=5, coef_mod=(-6, 6))
    s, pts = qd_data(402, s, synth.points(403, 20, 70, modulus_octaves=(-1, 0)))
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J)


def test_qd_results_beyond_double_double():
    """The same data rounded to double-double gives results that differ from
    the quad-double ones far above QD_TOL: the low parts are really used."""
    s = random_system(404, n=6, N=4, m=6, kmin=1, kmax=4, emax=4)
    s, pts = qd_data(405, s, synth.points(406, 6, 20))
    f, J = run_qd(s, pts)
    ef, ej = check_exact(s, pts, f, J)
    s2 = synth.System(s.n_vars, s.n_polys, s.poly_ptr, s.mono_ptr, s.pos, s.exp, s.coef[:, [0, 1, 4, 5]])
    ef2, _ = E.max_errors(s2, pts[..., [0, 1, 4, 5]], f, J, range(20))
    assert ef2 > 1e-40 > ef


def test_qd_gaussian_integers_exact():
    rng = np.random.Generator(np.random.PCG64(407))
    n = 5
    polys = []
    for _p in range(4):
        mons = []
        for _t in range(7):
            k = int(rng.integers(0, 5))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, 4, size=k).tolist()))
        polys.append(mons)
    s = synth.from_monomials(n, polys, synth.gaussian_int_cdd(rng, 28))
    P = 33
    pts = np.zeros((n, P, 8))
    pts[..., 0] = rng.integers(-2, 3, size=(n, P))
    pts[..., 4] = rng.integers(-2, 3, size=(n, P))
    f, J = run_qd(s, pts)
    for q in range(P):
        fx, Jx = E.evaluate_point(s, pts, q)
        for p in range(4):
            want = E.cx_to_dd(fx[p])
            assert (f[p, q, 0], f[p, q, 4]) == (want[0], want[2]) and want[1] == want[3] == 0.0
            assert np.all(f[p, q, [1, 2, 3, 5, 6, 7]] == 0.0)
            for i in range(n):
                w = E.cx_to_dd(Jx[p].get(i, E.ZERO))
                assert (J[p, i, q, 0], J[p, i, q, 4]) == (w[0], w[2])
                assert np.all(J[p, i, q, [1, 2, 3, 5, 6, 7]] == 0.0)


def test_qd_outputs_are_normalised():
    """Each part is at most half a unit in the last place of the part before
    it, and zero parts only follow zero parts."""
    s = random_system(408, n=10, N=6, m=12, kmin=1, kmax=6, emax=5, coef_mod=(-8, 8))
    s, pts = qd_data(409, s, synth.points(410, 10, 40, modulus_octaves=(-2, 2)))
    f, J = run_qd(s, pts)
    for arr in (f.reshape(-1, 8), J.reshape(-1, 8)):
        for c in (0, 4):
            parts = arr[:, c:c + 4]
            for i in range(3):
                hi, lo = parts[:, i], parts[:, i + 1]
                assert np.all(np.abs(lo) <= ulp(hi) / 2 + (hi == 0) * 0.0)
                assert np.all((hi != 0) | (lo == 0))


def test_qd_double_double_coefficients():
    """A system with double-double coefficients only (coef_qd NULL) at
    quad-double points: the coefficients are read with zero lower parts."""
    s = random_system(411, n=8, N=5, m=7, kmin=1, kmax=5, emax=4)
    rng = np.random.Generator(np.random.PCG64(412))
    pts = synth.widen_qd(rng, synth.points(413, 8, 21))
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J)


def test_qd_edge_cases_k0_k1_absent_variables():
    polys = [
        [([], []), ([0], [1]), ([1], [4])],
        [([0, 3], [1, 1]), ([1, 2], [2, 3])],
        [([], [])],
        [],
        [([2], [1]), ([0, 1, 2, 3], [1, 2, 1, 3]), ([], [])],
    ]
    M = sum(len(p) for p in polys)
    s = synth.from_monomials(5, polys, synth.random_cdd(np.random.Generator(np.random.PCG64(414)), M))
    s, pts = qd_data(415, s, synth.points(416, 5, 19))
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J)
    assert np.all(J[:, 4] == 0.0) and not np.any(np.signbit(J[:, 4]))
    assert np.all(J[2] == 0.0) and np.all(J[3] == 0.0)
    assert np.all(f[3] == 0.0)


def test_qd_zero_coordinates_and_wide_range():
    """Points with exact zero coordinates (products vanish) and moduli over
    2^-20 .. 2^20 (sums of terms of very different size)."""
    s = random_system(417, n=6, N=4, m=9, kmin=1, kmax=4, emax=4, coef_mod=(-30, 30))
    rng = np.random.Generator(np.random.PCG64(418))
    pts = synth.points(419, 6, 25, modulus_octaves=(-20, 20))
    pts[1, ::3] = 0.0
    s, pts = qd_data(420, s, pts)
    pts[1, ::3] = 0.0
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J)


def test_qd_largest_exponent():
    s = synth.from_monomials(3, [[([0, 1, 2], [256, 1, 3]), ([2], [255])], [([1], [2])]],
                             synth.random_cdd(np.random.Generator(np.random.PCG64(421)), 3))
    s, pts = qd_data(422, s, synth.points(423, 3, 17))
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J)


def test_qd_batch_of_uneven_systems():
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, points = [], []
    for i, (n, N, m, kmax, P) in enumerate([(7, 5, 6, 4, 19), (12, 3, 9, 6, 40), (4, 6, 3, 2, 0), (9, 9, 5, 5, 3)]):
        s = random_system(430 + i, n=n, N=N, m=m, kmin=1, kmax=kmax, emax=4)
        s, pts = qd_data(440 + i, s, synth.points(450 + i, n, P))
        systems.append(s)
        points.append(pts)
    many = pkg.PolyEvalMany(systems, [p.shape[1] for p in points], pkg.PE_QD_INT)
    fs, Js = many.eval([to_device(p) for p in points])
    torch.cuda.synchronize()
    for s, pts, f, J in zip(systems, points, fs, Js):
        if pts.shape[1]:
            check_exact(s, pts, f.cpu().numpy(), J.cpu().numpy())


def test_qd_deterministic_chunks_and_autotune():
    """Repeated calls give identical bits; the autotuned launch (another
    chunk count or launch shape) stays within the tolerance."""
    import torch

    import paper_1201_0499_gb300 as pkg

    s = random_system(460, n=16, N=16, m=24, kmin=2, kmax=6, emax=4)
    s, pts = qd_data(461, s, synth.points(462, 16, 48))
    ev = pkg.PolyEval(s, pkg.PE_QD_INT, max_points=48)
    x = to_device(pts)
    f1, J1 = ev.eval(x)
    f2, J2 = ev.eval(x)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2) and torch.equal(J1, J2)
    chunks, shape, groups = ev.autotune(x)
    assert chunks in (1, 2, 4, 8) and shape in (1, 2) and groups == 1
    f3, J3 = ev.eval(x)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    check_exact(s, pts, f3.cpu().numpy(), J3.cpu().numpy(), points_idx=[0, 17, 47])


def test_qd_config2_sampled():
    """The benchmark workload (n = 32, m = 64, k = 9, 1024 points) with
    quad-double data, at the launch the benchmark uses: sampled points and
    polynomials against the exact oracle."""
    s, pts = synth.config(2)
    s, pts = qd_data(470, s, pts)
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J, points_idx=[0, 511, 1023], polys=[0, 13, 31])


def test_qd_config3_sampled_and_euler_identity():
    """n = 64, m = 256, k = 16, 4096 points (config 3) with quad-double data:
    sampled outputs against the exact oracle; on the homogeneous variant
    (degree 24) Euler's identity sum_i x_i df/dx_i = 24 f checked exactly at
    sampled points, within the quad-double tolerance."""
    from fractions import Fraction

    s, pts = synth.config(3)
    s, pts = qd_data(471, s, pts)
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J, points_idx=[0, 4095], polys=[0, 63])
    s, pts = synth.config(3, homogeneous=True)
    s, pts = qd_data(472, s, pts)
    f, J = run_qd(s, pts)

    def fr(v):
        return sum(Fraction(float(x)) for x in v[:4]), sum(Fraction(float(x)) for x in v[4:])

    for q in (0, 4095):
        for p in (0, 40):
            lr, li = Fraction(0), Fraction(0)
            for i in range(s.n_vars):
                xr, xi = fr(pts[i, q])
                jr, ji = fr(J[p, i, q])
                lr += xr * jr - xi * ji
                li += xr * ji + xi * jr
            ffr, ffi = fr(f[p, q])
            res = abs(complex(float(lr - 24 * ffr), float(li - 24 * ffi)))
            Sf, _ = E.scales_point(s, pts, q, polys=[p])
            assert res <= 48 * QD_TOL * Sf[p], (q, p, res / Sf[p])


def test_qd_config4_ragged_batch_sampled():
    """The 200 uneven systems of config 4 in one launch, quad-double data:
    sampled systems and points against the exact oracle."""
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, pts = synth.config(4)
    rng = np.random.Generator(np.random.PCG64(473))
    qs = [s.to_qd(474 + i) for i, s in enumerate(systems)]
    qp = [synth.widen_qd(rng, p) for p in pts]
    ev = pkg.PolyEvalMany(qs, [p.shape[1] for p in qp], pkg.PE_QD_INT)
    fs, Js = ev.eval([to_device(p) for p in qp])
    torch.cuda.synchronize()
    assert pkg.polyeval_status(ev.handle) == pkg.PE_OK
    for si in rng.choice(len(systems), size=5, replace=False):
        P = qp[si].shape[1]
        if P == 0:
            continue
        q = [0, P - 1] if P > 1 else [0]
        polys = sorted({0, qs[si].n_polys - 1})
        check_exact(qs[si], qp[si], fs[si].cpu().numpy(), Js[si].cpu().numpy(), points_idx=q, polys=polys)


def test_qd_config5_sampled():
    """n = 128, m = 1024, k = 32 (config 5) at 2048 of its points, quad-double
    data: a sampled output row against the exact oracle."""
    s, pts = synth.config(5, n_points=2048)
    s, pts = qd_data(475, s, pts)
    f, J = run_qd(s, pts)
    check_exact(s, pts, f, J, points_idx=[2047], polys=[127])


def test_qd_rejects_paper_kernels():
    import paper_1201_0499_gb300 as pkg

    s = random_system(480, n=4, N=4, m=3, kmin=3, kmax=3, emax=2)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.PolyEval(s, pkg.PE_QD_INT, max_points=4, flags=pkg.PE_PAPER_KERNELS)
    assert e.value.code == pkg.PE_EINVAL
