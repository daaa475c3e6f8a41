"""polyeval_eval_noalloc, the entry point for callers that cannot let the
library allocate device memory (their memory belongs to another allocator or
to a fixed arena): the system, points and outputs live in the caller's own
device buffers, and the only scratch is the library's static device array.

Checked through the C ABI against polyeval_eval (which allocates at create
time) on two calls in a row, within the double-double tolerance the other
tests use.  Kept in a file of its own that pytest collects last.
"""
import numpy as np
import pytest

import synth

from _util import DD_TOL, normwise_vs, scales

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


def _device_system(torch, system):
    """The caller's own device copies of the system arrays, and a pe_system
    whose pointer fields hold their device addresses."""
    import paper_1201_0499_gb300 as pkg

    arrays = [
        torch.from_numpy(np.ascontiguousarray(system.poly_ptr, dtype=np.int64)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.mono_ptr, dtype=np.int64)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.pos, dtype=np.int32)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.exp, dtype=np.int32)).cuda(),
        torch.from_numpy(np.ascontiguousarray(system.coef, dtype=np.float64)).cuda(),
    ]
    ds = pkg.pe_system(system.n_vars, system.n_polys, *[a.data_ptr() for a in arrays])
    return ds, arrays


def test_noalloc_matches_eval_on_two_calls(torch_cuda):
    torch = torch_cuda
    import paper_1201_0499_gb300 as pkg

    system, _ = synth.config(2, n_points=1)
    n, N = system.n_vars, system.n_polys
    P = 200  # 13 tiles of 16 points, the last one ragged
    max_k = int(np.diff(system.mono_ptr).max())
    max_exp = int(system.exp.max())
    ds, keep = _device_system(torch, system)
    ref = pkg.PolyEval(system, pkg.PE_DD, max_points=P)
    for call, seed in enumerate((501, 502)):
        pts = synth.points(seed, n, P)
        x = torch.from_numpy(pts).cuda()
        f = torch.full((N, P, 4), float("nan"), dtype=torch.float64, device="cuda")
        J = torch.full((N, n, P, 4), float("nan"), dtype=torch.float64, device="cuda")
        pkg.polyeval_eval_noalloc(ds, max_k, max_exp, x, P, f, J)
        f_ref, J_ref = ref.eval(x)
        torch.cuda.synchronize()
        Sf, SJ = scales(system, pts)
        assert normwise_vs(f.cpu().numpy(), f_ref.cpu().numpy(), Sf) <= DD_TOL, call
        assert normwise_vs(J.cpu().numpy(), J_ref.cpu().numpy(), SJ) <= DD_TOL, call
    ref.close()
    del keep


def test_noalloc_rejects_sizes_beyond_the_scratch(torch_cuda):
    torch = torch_cuda
    import paper_1201_0499_gb300 as pkg

    system, _ = synth.config(2, n_points=1)
    ds, keep = _device_system(torch, system)
    x = torch.zeros((32, 8, 4), dtype=torch.float64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # (max_exp - 2) * n * P complex double-doubles must fit in 16 MiB (524288 of them)
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 9, 5, x, 6000, out, out)
    assert e.value.code == pkg.PE_ERANGE
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 300, 5, x, 8, out, out)
    assert e.value.code == pkg.PE_ERANGE
    with pytest.raises(pkg.PolyEvalError) as e:
        pkg.polyeval_eval_noalloc(ds, 9, 5, 0, 8, out, out)
    assert e.value.code == pkg.PE_EINVAL
    del keep


def _run_noalloc(torch, system, pts, max_k, max_exp, ds=None):
    import paper_1201_0499_gb300 as pkg

    keep = None
    if ds is None:
        ds, keep = _device_system(torch, system)
    n, N, P = system.n_vars, system.n_polys, pts.shape[1]
    x = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    f = torch.full((N, P, 4), float("nan"), dtype=torch.float64, device="cuda")
    J = torch.full((N, n, P, 4), float("nan"), dtype=torch.float64, device="cuda")
    pkg.polyeval_eval_noalloc(ds, max_k, max_exp, x, P, f, J)
    torch.cuda.synchronize()
    del keep
    return f.cpu().numpy(), J.cpu().numpy()


def test_noalloc_against_the_oracles(torch_cuda):
    """Every output of 200 points (13 tiles, the last one ragged) of the
    n = 32, m = 64, k = 9 system against the C double-double oracle, and
    sampled outputs against the exact oracle (Section 2, Eq. 1)."""
    import oracle
    from oracle import exact as E

    system, _ = synth.config(2, n_points=1)
    pts = synth.points(503, system.n_vars, 200)
    f, J = _run_noalloc(torch_cuda, system, pts, int(np.diff(system.mono_ptr).max()), int(system.exp.max()))
    Fo, Jo = oracle.dd_eval(system, pts, threads=0)
    Sf, SJ = scales(system, pts)
    assert normwise_vs(f, Fo, Sf) <= DD_TOL
    assert normwise_vs(J, Jo, SJ) <= DD_TOL
    ef, ej = E.max_errors(system, pts, f, J, [0, 199], polys=[0, 31])
    assert ef <= DD_TOL and ej <= DD_TOL, (ef, ej)


def _small_system(seed, n, N, m, kmin, kmax, emax):
    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _p in range(N):
        mons = []
        for _t in range(m):
            k = int(rng.integers(kmin, kmax + 1))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, emax + 1, size=k).tolist()))
        polys.append(mons)
    return synth.from_monomials(n, polys, synth.random_cdd(rng, N * m))


@pytest.mark.parametrize("emax", [1, 2])
def test_noalloc_without_power_table_and_k_0_1_2(torch_cuda, emax):
    """Exponents at most 1 or 2 (no power table: a = 2 reads the point),
    constant terms and monomials of one and two variables, 37 points; every
    output against the exact oracle.  The second run passes max_k = 256 (the
    largest bound) for the same system."""
    from oracle import exact as E

    system = _small_system(504 + emax, n=7, N=5, m=9, kmin=0, kmax=2, emax=emax)
    assert int(np.diff(system.mono_ptr).min()) == 0
    pts = synth.points(506, 7, 37, modulus_octaves=(-1, 0))
    for max_k in (2, 256):
        f, J = _run_noalloc(torch_cuda, system, pts, max_k, emax)
        ef, ej = E.max_errors(system, pts, f, J, range(37))
        assert ef <= DD_TOL and ej <= DD_TOL, (max_k, ef, ej)


@pytest.mark.parametrize("fault", ["position_n", "exponent_above_max", "k_above_max"])
def test_noalloc_bad_metadata_flags_f_as_nan(torch_cuda, fault):
    """Metadata that breaks the caller's stated limits, in device memory: a
    variable position equal to n, an exponent above max_exp, a monomial with
    more variables than max_k.  The kernel checks every entry before any load
    through it, skips that monomial and writes f of its polynomial as NaN;
    the other polynomials stay within the tolerance of the exact oracle."""
    torch = torch_cuda
    from oracle import exact as E

    rng = np.random.Generator(np.random.PCG64(507))
    n, N, m = 6, 4, 5
    polys = [[(sorted(rng.choice(n, size=int(rng.integers(1, 4)), replace=False).tolist()), None)
              for _t in range(m)] for _p in range(N)]
    polys = [[(pos, rng.integers(1, 4, size=len(pos)).tolist()) for pos, _ in mons] for mons in polys]
    bad_poly = 2
    polys[bad_poly].append(([0, 2, 3, 5], [1, 2, 1, 3]))  # the only monomial with 4 variables
    M = sum(len(mons) for mons in polys)
    system = synth.from_monomials(n, polys, synth.random_cdd(rng, M))
    pts = synth.points(508, n, 21)
    max_k, max_exp = 4, 3
    t = int(system.poly_ptr[bad_poly + 1]) - 1  # the appended monomial
    a, b = int(system.mono_ptr[t]), int(system.mono_ptr[t + 1])
    pos, exp = system.pos.copy(), system.exp.copy()
    if fault == "position_n":
        pos[b - 1] = n
    elif fault == "exponent_above_max":
        exp[a] = max_exp + 1
    else:
        max_k = 3
    bad = synth.System(n, N, system.poly_ptr, system.mono_ptr, pos, exp, system.coef)
    ds, keep = _device_system(torch, bad)
    f, J = _run_noalloc(torch, bad, pts, max_k, max_exp, ds=ds)
    del keep
    assert np.all(np.isnan(f[bad_poly, :, 0]))
    good = [p for p in range(N) if p != bad_poly]
    ef, ej = E.max_errors(system, pts, f, J, range(21), polys=good)
    assert ef <= DD_TOL and ej <= DD_TOL, (ef, ej)
    assert not np.any(np.isnan(f[good]))
