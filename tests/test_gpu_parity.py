"""Parity of the CUDA path with the oracle (complex double-double and complex
double), on small cases element by element and on the full-size workloads by
sampled outputs.

Tolerances (normwise, see tests/_util.py): 1e-28 for double-double and 1e-13
for double.  Gaussian-integer inputs whose results stay below 2**53 must come
out bit-exact in both precisions.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import DD_TOL, F64_TOL, PRECS, fp64_inputs, normwise_vs, run, scales, to_device, tol

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1201_0499_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(0)


def check_exact_oracle(system, pts, f, J, tol, points_idx=None, polys=None, dd=True):
    if not dd:
        system, pts = fp64_inputs(system, pts)
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


# ----------------------------------------------------------------------------
# small cases: every output against the exact oracle
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_several_tiles_ragged_tail(prec):
    s = random_system(101, n=20, N=12, m=10, kmin=1, kmax=7, emax=5, coef_mod=(-6, 6))
    pts = synth.points(102, 20, 70, modulus_octaves=(-1, 0))  # 5 tiles of 16, last one ragged
    f, J = run(s, pts, prec)
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")


@pytest.mark.parametrize("prec", PRECS)
def test_gaussian_integers_bit_exact(prec):
    rng = np.random.Generator(np.random.PCG64(103))
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
    pts = np.zeros((n, P, 4))
    pts[..., 0] = rng.integers(-2, 3, size=(n, P))
    pts[..., 2] = rng.integers(-2, 3, size=(n, P))
    f, J = run(s, pts, prec)
    Fx, Jx = E.evaluate_dd(s, pts, range(P))
    assert np.array_equal(f, Fx)
    assert np.array_equal(J, Jx)


@pytest.mark.parametrize("prec", PRECS)
def test_worked_example_common_factor(prec):
    """x1^3 x2^7 x3^2 (Section 3.1): common factor x1^2 x2^6 x3; the
    derivatives are 3 x1^2 x2^7 x3^2, 7 x1^3 x2^6 x3^2 and 2 x1^3 x2^7 x3."""
    s = synth.from_monomials(3, [[([0, 1, 2], [3, 7, 2])]], [[1.0, 0, 0, 0]])
    pts = np.zeros((3, 2, 4))
    pts[:, 0, 0] = [2, -1, 3]
    pts[:, 0, 2] = [1, 1, 0]
    pts[:, 1] = synth.points(104, 3, 1)[:, 0]
    f, J = run(s, pts, prec)
    x = [complex(2, 1), complex(-1, 1), complex(3, 0)]
    want_f = x[0] ** 3 * x[1] ** 7 * x[2] ** 2
    want_J = [3 * x[0] ** 2 * x[1] ** 7 * x[2] ** 2, 7 * x[0] ** 3 * x[1] ** 6 * x[2] ** 2,
              2 * x[0] ** 3 * x[1] ** 7 * x[2]]
    assert (f[0, 0, 0], f[0, 0, 2]) == (want_f.real, want_f.imag)
    for i in range(3):
        assert (J[0, i, 0, 0], J[0, i, 0, 2]) == (want_J[i].real, want_J[i].imag)
        assert J[0, i, 0, 1] == 0.0 and J[0, i, 0, 3] == 0.0
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")


@pytest.mark.parametrize("prec", PRECS)
def test_edge_cases_k0_k1_k2_absent_variables(prec):
    # constant terms, k = 1 and k = 2 monomials, a variable (x4) in no monomial,
    # a polynomial with only a constant, an empty polynomial
    polys = [
        [([], []), ([0], [1]), ([1], [4])],
        [([0, 3], [1, 1]), ([1, 2], [2, 3])],
        [([], [])],
        [],
        [([2], [1]), ([0, 1, 2, 3], [1, 2, 1, 3]), ([], [])],
    ]
    M = sum(len(p) for p in polys)
    s = synth.from_monomials(5, polys, synth.random_cdd(np.random.Generator(np.random.PCG64(105)), M))
    pts = synth.points(106, 5, 19)
    f, J = run(s, pts, prec)
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")
    assert np.all(J[:, 4] == 0.0)              # x4 occurs nowhere
    assert not np.any(np.signbit(J[:, 4]))      # written as +0.0
    assert np.all(J[2] == 0.0) and np.all(J[3] == 0.0)
    assert np.all(f[3] == 0.0)


@pytest.mark.parametrize("prec", PRECS)
def test_one_variable_and_one_point(prec):
    s = synth.from_monomials(1, [[([0], [5]), ([], [])]], [[0.5, 0, -2, 0], [1, 0, 0, 0]])
    pts = synth.points(107, 1, 1)
    f, J = run(s, pts, prec)
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")


@pytest.mark.parametrize("prec", PRECS)
def test_largest_exponent_and_variable_index(prec):
    """Exponent 256 (the largest the paper's byte encoding allows) and the
    variable index n-1 = 65534 (the largest position)."""
    n = 65535
    s = synth.from_monomials(n, [[([0, 1000, n - 1], [256, 1, 3]), ([n - 1], [255])], [([n - 2], [2])]],
                             synth.random_cdd(np.random.Generator(np.random.PCG64(108)), 3))
    P = 17
    pts = np.zeros((n, P, 4))
    used = [0, 1000, n - 2, n - 1]
    pts[used] = synth.points(110, len(used), P)  # unit circle: |x|^256 stays near 1
    f, J = run(s, pts, prec)
    s_ref, p_ref = (s, pts) if prec != "f64" else fp64_inputs(s, pts)
    tl = tol(prec)
    for q in range(P):
        fx, Jx = E.evaluate_point(s_ref, p_ref, q)
        Sf, SJ = E.scales_point(s_ref, p_ref, q)
        for p in range(2):
            assert E.normwise_error(f[p, q], fx[p], Sf[p]) <= tl
            for i, v in Jx[p].items():
                assert E.normwise_error(J[p, i, q], v, SJ[p][i]) <= tl
    mask = np.ones(n, dtype=bool)
    mask[[0, 1000, n - 1]] = False
    assert np.all(J[0][mask] == 0.0)
    mask = np.ones(n, dtype=bool)
    mask[n - 2] = False
    assert np.all(J[1][mask] == 0.0)


def test_empty_inputs():
    import torch

    import paper_1201_0499_gb300 as pkg

    s = random_system(111, n=6, N=3, m=4, kmin=1, kmax=3, emax=3)
    ev = pkg.PolyEval(s, pkg.PE_DD, max_points=8)
    x = torch.zeros((6, 0, 4), dtype=torch.float64, device="cuda")
    f, J = ev.eval(x)
    assert f.shape == (3, 0, 4) and J.shape == (3, 6, 0, 4)
    # no polynomials at all
    e = synth.from_monomials(4, [], np.zeros((0, 4)))
    ev2 = pkg.PolyEval(e, pkg.PE_DD, max_points=4)
    f2, J2 = ev2.eval(to_device(synth.points(112, 4, 4)))
    assert f2.numel() == 0 and J2.numel() == 0
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK


def test_argument_errors():
    import torch

    import paper_1201_0499_gb300 as pkg

    s = random_system(113, n=4, N=2, m=3, kmin=1, kmax=2, emax=2)
    ev = pkg.PolyEval(s, pkg.PE_DD, max_points=8)
    x = to_device(synth.points(114, 4, 9))
    with pytest.raises(pkg.PolyEvalError) as e:
        ev.eval(x)  # 9 > max_points
    assert e.value.code == pkg.PE_ERANGE
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval(ev.handle, 0, 4, 0, 0)
    assert e.value.code == pkg.PE_EINVAL
    bad = synth.from_monomials(4, [[([1, 0], [1, 1])]], [[1, 0, 0, 0]])
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.PolyEval(bad, pkg.PE_DD, max_points=4)
    assert e.value.code == pkg.PE_EINVAL
    with pytest.raises(pkg.PolyEvalError):
        pkg.polyeval_create(s, 7, 0, 4)
    with pytest.raises(pkg.PolyEvalError):
        pkg.polyeval_create(s, pkg.PE_DD, 0, 0)
    # device arrays must be 16-byte aligned (vector accesses): rejected on the host
    x8 = to_device(synth.points(114, 4, 8))
    f = torch.empty((2, 8, 4), dtype=torch.float64, device="cuda")
    J = torch.empty((2, 4, 8, 4), dtype=torch.float64, device="cuda")
    for args in ((x8.data_ptr() + 8, f.data_ptr(), J.data_ptr()), (x8.data_ptr(), f.data_ptr() + 8, J.data_ptr()),
                 (x8.data_ptr(), f.data_ptr(), J.data_ptr() + 8)):
        with pytest.raises(pkg.PolyEvalError) as e:
            pkg.polyeval_eval(ev.handle, args[0], 7, args[1], args[2])
        assert e.value.code == pkg.PE_EINVAL


def test_deterministic_and_host_entry_point_agree():
    import torch

    import paper_1201_0499_gb300 as pkg

    s, pts = synth.config(2, n_points=100)
    ev = pkg.PolyEval(s, pkg.PE_DD, max_points=100)
    x = to_device(pts)
    f1, J1 = ev.eval(x)
    f2, J2 = ev.eval(x)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2) and torch.equal(J1, J2)
    hf = torch.empty(f1.shape, dtype=torch.float64).pin_memory()
    hJ = torch.empty(J1.shape, dtype=torch.float64).pin_memory()
    hp = torch.from_numpy(pts).pin_memory()
    pkg.polyeval_eval_host(ev.handle, hp, 100, hf, hJ)
    assert torch.equal(hf, f1.cpu()) and torch.equal(hJ, J1.cpu())


def test_cuda_graph_replay_matches_eager():
    import torch

    import paper_1201_0499_gb300 as pkg

    s, pts = synth.config(2, n_points=64)
    ev = pkg.PolyEval(s, pkg.PE_DD, max_points=64)
    x = to_device(pts)
    f_ref, J_ref = ev.eval(x)
    torch.cuda.synchronize()
    f = torch.empty_like(f_ref)
    J = torch.empty_like(J_ref)
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        ev.eval(x, f, J)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        ev.eval(x, f, J)
    f.zero_()
    J.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(f, f_ref) and torch.equal(J, J_ref)


# ----------------------------------------------------------------------------
# the five workloads
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_config1_tiny(prec):
    s, pts = synth.config(1)
    f, J = run(s, pts, prec)
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")


@pytest.mark.parametrize("prec", ["dd", "ddint"])
def test_config2_full_batch_dd(prec):
    """The benchmark workload at full size (1024 points): every output
    against the C double-double oracle (itself within 1e-30 of exact), and
    sampled points against the exact oracle."""
    import oracle

    s, pts = synth.config(2)
    f, J = run(s, pts, prec)
    Fo, Jo = oracle.dd_eval(s, pts, threads=0)
    Sf, SJ = scales(s, pts)
    assert normwise_vs(f, Fo, Sf) <= DD_TOL
    assert normwise_vs(J, Jo, SJ) <= DD_TOL
    check_exact_oracle(s, pts, f, J, DD_TOL, points_idx=[0, 511, 1023], polys=[0, 13, 31])


def test_config2_full_batch_f64():
    s, pts = synth.config(2)
    f, J = run(s, pts, False)
    s64, p64 = fp64_inputs(s, pts)
    check_exact_oracle(s64, p64, f, J, F64_TOL, points_idx=[0, 700, 1023], polys=[0, 31])


@pytest.mark.parametrize("prec", ["dd", "ddint"])
def test_config3_homogeneous_euler_identity(prec):
    """sum_i x_i df_p/dx_i = 24 f_p on the homogeneous variant (degree 24),
    checked exactly on sampled points; and the outputs against the exact
    oracle there."""
    s, pts = synth.config(3, homogeneous=True)
    f, J = run(s, pts, prec)
    from fractions import Fraction

    for q in (0, 2047, 4095):
        for p in (0, 40):
            lhs = [Fraction(0), Fraction(0)]
            for i in range(s.n_vars):
                xr = Fraction(pts[i, q, 0]) + Fraction(pts[i, q, 1])
                xi = Fraction(pts[i, q, 2]) + Fraction(pts[i, q, 3])
                jr = Fraction(J[p, i, q, 0]) + Fraction(J[p, i, q, 1])
                ji = Fraction(J[p, i, q, 2]) + Fraction(J[p, i, q, 3])
                lhs[0] += xr * jr - xi * ji
                lhs[1] += xr * ji + xi * jr
            fr = Fraction(f[p, q, 0]) + Fraction(f[p, q, 1])
            fi = Fraction(f[p, q, 2]) + Fraction(f[p, q, 3])
            res = abs(complex(float(lhs[0] - 24 * fr), float(lhs[1] - 24 * fi)))
            Sf, _ = E.scales_point(s, pts, q, polys=[p])
            assert res <= 48 * DD_TOL * Sf[p], (q, p, res / Sf[p])
    check_exact_oracle(s, pts, f, J, DD_TOL, points_idx=[1], polys=[5])


@pytest.mark.parametrize("prec", ["dd", "ddint"])
def test_config4_ragged_batch(prec):
    import torch

    import oracle
    import paper_1201_0499_gb300 as pkg

    systems, pts = synth.config(4)
    ev = pkg.PolyEvalMany(systems, [p.shape[1] for p in pts], pkg.PE_DD if prec == "dd" else pkg.PE_DD_INT)
    fs, Js = ev.eval([to_device(p) for p in pts])
    torch.cuda.synchronize()
    assert pkg.polyeval_status(ev.handle) == pkg.PE_OK
    rng = np.random.Generator(np.random.PCG64(115))
    # the smallest systems in full against the C oracle
    order = np.argsort([s.n_monos * p.shape[1] for s, p in zip(systems, pts)])
    for si in order[:6]:
        s, x = systems[si], pts[si]
        f, J = fs[si].cpu().numpy(), Js[si].cpu().numpy()
        Fo, Jo = oracle.dd_eval(s, x, threads=0)
        Sf, SJ = scales(s, x)
        assert normwise_vs(f, Fo, Sf) <= DD_TOL, si
        assert normwise_vs(J, Jo, SJ) <= DD_TOL, si
    # sampled outputs of other systems against the exact oracle
    for si in rng.choice(len(systems), size=5, replace=False):
        s, x = systems[si], pts[si]
        f, J = fs[si].cpu().numpy(), Js[si].cpu().numpy()
        q = int(rng.integers(0, x.shape[1]))
        p = int(rng.integers(0, s.n_polys))
        check_exact_oracle(s, x, f, J, DD_TOL, points_idx=[q], polys=[p])


# ----------------------------------------------------------------------------
# bounds and chunking
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("prec", PRECS)
def test_outputs_do_not_touch_guard_bands(prec):
    """f and J written through views inside larger buffers filled with a
    canary: nothing outside the views changes (no out-of-bounds stores,
    including the lanes past a ragged tail and the chunk scratch)."""
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import pe_precision

    s = random_system(121, n=9, N=7, m=6, kmin=0, kmax=4, emax=4)
    for P in (1, 5, 17, 40):
        pts = synth.points(122 + P, 9, P)
        dd = prec != "f64"
        c = 4 if dd else 2
        x = to_device(pts, dd)
        guard = 1000
        canary = -1.2345e300
        fbuf = torch.full((7 * P * c + 2 * guard,), canary, dtype=torch.float64, device="cuda")
        Jbuf = torch.full((7 * 9 * P * c + 2 * guard,), canary, dtype=torch.float64, device="cuda")
        f = fbuf[guard:guard + 7 * P * c].view(7, P, c)
        J = Jbuf[guard:guard + 7 * 9 * P * c].view(7, 9, P, c)
        ev = pkg.PolyEval(s if dd else s.as_fp64(), pe_precision(prec), max_points=P)
        ev.eval(x, f, J)
        torch.cuda.synchronize()
        assert ev.status() == pkg.PE_OK
        for buf in (fbuf, Jbuf):
            assert torch.all(buf[:guard] == canary) and torch.all(buf[-guard:] == canary)
        assert not torch.any(f == canary) and not torch.any(J == canary)
        fo, Jo = f.cpu().numpy(), J.cpu().numpy()
        if not dd:
            from _util import widen

            fo, Jo = widen(fo), widen(Jo)
        check_exact_oracle(s, pts, fo, Jo, tol(prec), dd=dd)


@pytest.mark.parametrize("prec", PRECS)
def test_more_chunks_than_monomials(prec):
    """One point and polynomials of 1..3 monomials: the call splits the
    monomials into up to 8 chunks, most of them empty."""
    s = random_system(123, n=4, N=3, m=2, kmin=1, kmax=3, emax=3)
    pts = synth.points(124, 4, 1)
    f, J = run(s, pts, prec)
    check_exact_oracle(s, pts, f, J, tol(prec), dd=prec != "f64")


def test_integer_path_deterministic_and_close_to_fp64_dd():
    import torch

    import paper_1201_0499_gb300 as pkg

    s, pts = synth.config(2, n_points=200)
    x = to_device(pts)
    a = pkg.PolyEval(s, pkg.PE_DD_INT, max_points=200)
    f1, J1 = a.eval(x)
    f2, J2 = a.eval(x)
    torch.cuda.synchronize()
    assert torch.equal(f1, f2) and torch.equal(J1, J2)
    b = pkg.PolyEval(s, pkg.PE_DD, max_points=200)
    f3, J3 = b.eval(x)
    torch.cuda.synchronize()
    Sf, SJ = scales(s, pts)
    assert normwise_vs(f1.cpu().numpy(), f3.cpu().numpy(), Sf) <= 2 * DD_TOL
    assert normwise_vs(J1.cpu().numpy(), J3.cpu().numpy(), SJ) <= 2 * DD_TOL


@pytest.mark.parametrize("prec", ["dd", "ddint"])
def test_autotune_then_eval(prec):
    """The autotuner's choice is kept for the point count and gives results
    within the double-double tolerance of the exact oracle."""
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import pe_precision

    s, pts = synth.config(2, n_points=300)
    ev = pkg.PolyEval(s, pe_precision(prec), max_points=300)
    x = to_device(pts)
    chunks, shape, groups = ev.autotune(x)
    assert chunks in (1, 2, 4, 8) and shape in (1, 2) and groups == 1  # 300 points: no groups tried
    f, J = ev.eval(x)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    check_exact_oracle(s, pts, f.cpu().numpy(), J.cpu().numpy(), DD_TOL, points_idx=[0, 299], polys=[0, 31])


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_set_launch_every_choice(prec):
    """Every launch a caller can fix with polyeval_set_launch (chunks 1..8,
    both shapes) gives the same outputs up to the summation order of the
    chunks, within the tolerance of the exact oracle at sampled points."""
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import QD_TOL, pe_precision

    s, pts = synth.config(2, n_points=100)
    if prec == "qd":
        rng = np.random.Generator(np.random.PCG64(116))
        s, pts = s.to_qd(117), synth.widen_qd(rng, pts)
    ev = pkg.PolyEval(s, pe_precision(prec), max_points=100)
    x = to_device(pts)
    for chunks in (1, 3, 8):
        for shape in (1, 2):
            pkg.polyeval_set_launch(ev.handle, 100, chunks, shape)
            f, J = ev.eval(x)
            torch.cuda.synchronize()
            assert ev.status() == pkg.PE_OK
            check_exact_oracle(s, pts, f.cpu().numpy(), J.cpu().numpy(), QD_TOL if prec == "qd" else DD_TOL,
                               points_idx=[0, 99], polys=[5])
    pkg.polyeval_set_launch(ev.handle, 100, 0, 0)  # back to the built-in choice
    with pytest.raises(pkg.PolyEvalError):
        pkg.polyeval_set_launch(ev.handle, 100, 9, 1)


@pytest.mark.parametrize("prec", ["dd", "f64"])
@pytest.mark.parametrize("P", [1, 3, 5, 15])
def test_monomial_groups_few_points(prec, P):
    """Few points: G monomial groups per warp (32 / G lanes per monomial).
    Monomials of different k in one polynomial make the groups of a round
    diverge; two monomials of a round may share variables.  Every G against
    the exact oracle, every output."""
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import pe_precision

    s = random_system(118, n=10, N=5, m=23, kmin=0, kmax=6, emax=4)
    pts = synth.points(119, 10, P)
    if prec == "f64":
        s64, p64 = fp64_inputs(s, pts)
    ev = pkg.PolyEval(s if prec == "dd" else s.as_fp64(), pe_precision(prec), max_points=P)
    x = to_device(pts, prec == "dd")
    for G in (1, 2, 4, 8, 16):
        for chunks in (1, 3):
            pkg.polyeval_set_launch(ev.handle, P, chunks, 0, G)
            f, J = ev.eval(x)
            torch.cuda.synchronize()
            assert ev.status() == pkg.PE_OK
            f, J = f.cpu().numpy(), J.cpu().numpy()
            if prec == "f64":
                from _util import widen

                f, J = widen(f), widen(J)
            check_exact_oracle(s, pts, f, J, tol(prec), dd=prec == "dd")
    g = ev.autotune(x)[2]
    assert g in (1, 2, 4, 8, 16)


@pytest.mark.parametrize("prec,P", [("dd", 6200), ("ddint", 4101), ("f64", 8200)])
def test_host_entry_point_in_chunks_matches_device(prec, P):
    """polyeval_eval_host on outputs above 512 MiB splits the points into
    chunks (here 3 chunks of 2067/2067/2066 points, 2 of 2051/2050, 2 of 4100) and
    copies each chunk's columns to the host while the next is evaluated:
    bit-identical to polyeval_eval on the device (each point's sums run in
    monomial order whatever tile holds it)."""
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import pe_precision

    s, _ = synth.config(3, n_points=1)
    pts = synth.points(132, s.n_vars, P, modulus_octaves=(-1, 0))
    dd = prec != "f64"
    sy = s if dd else s.as_fp64()
    host_pts = np.ascontiguousarray(pts if dd else pts[..., [0, 2]])
    c = host_pts.shape[-1]
    ev = pkg.PolyEval(sy, pe_precision(prec), max_points=P)
    f_dev, J_dev = ev.eval(torch.from_numpy(host_pts).cuda())
    torch.cuda.synchronize()
    hp = torch.from_numpy(host_pts).pin_memory()
    hf = torch.full((s.n_polys, P, c), float("nan"), dtype=torch.float64).pin_memory()
    hJ = torch.full((s.n_polys, s.n_vars, P, c), float("nan"), dtype=torch.float64).pin_memory()
    for _ in range(2):  # the second call reuses the staging buffers and the handle's copy stream
        pkg.polyeval_eval_host(ev.handle, hp, P, hf, hJ)
        assert torch.equal(hf, f_dev.cpu()) and torch.equal(hJ, J_dev.cpu())
        hf.fill_(float("nan"))
        hJ.fill_(float("nan"))
    assert ev.status() == pkg.PE_OK
    ev.close()
