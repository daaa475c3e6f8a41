"""Batches of uneven systems in one launch (polyeval_eval_many) under every
launch a caller can fix, and the batch autotuner: monomial chunks of every
(polynomial, tile) item, the launch shape, and the monomial groups of a
system's partial last tile.  Every output of a small batch against the exact
oracle (Section 2, Eq. 1); the 200-system workload after autotuning against
the C double-double oracle in full on its six smallest systems and against
the exact oracle at sampled outputs.
"""
import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import DD_TOL, fp64_inputs, normwise_vs, pe_precision, scales, to_device, tol, widen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1201_0499_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(0)


def _random_system(seed, n, N, m, kmin, kmax, emax):
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


def _small_batch(prec):
    """Six systems: partial tiles of 1, 3, 5 and 15 points, a system with no
    points, two full tiles and a ragged tail; k = 0 .. 6 within a polynomial."""
    shapes = [(6, 4, 9, 0, 5, 1), (9, 5, 7, 1, 6, 3), (4, 3, 5, 0, 3, 0), (11, 6, 8, 2, 6, 37), (5, 5, 6, 0, 4, 15),
              (7, 3, 10, 1, 5, 5)]
    systems, points = [], []
    rng = np.random.Generator(np.random.PCG64(603))
    for i, (n, N, m, kmin, kmax, P) in enumerate(shapes):
        s = _random_system(600 + i, n, N, m, kmin, kmax, 4)
        x = synth.points(610 + i, n, P, modulus_octaves=(-1, 0))
        if prec == "qd":
            s, x = s.to_qd(620 + i), synth.widen_qd(rng, x)
        systems.append(s)
        points.append(x)
    return systems, points


def _device_points(prec, x):
    if prec == "f64":
        return to_device(x, False)
    return to_device(x)


def _check_batch(prec, systems, points, fs, Js):
    for s, x, f, J in zip(systems, points, fs, Js):
        if x.shape[1] == 0:
            continue
        f, J = f.cpu().numpy(), J.cpu().numpy()
        if prec == "f64":
            f, J = widen(f), widen(J)
            s, x = fp64_inputs(s, x)
        ef, ej = E.max_errors(s, x, f, J, range(x.shape[1]))
        assert ef <= tol(prec) and ej <= tol(prec), (ef, ej)


@pytest.mark.parametrize("prec", ["dd", "f64", "ddint", "qd"])
def test_batch_every_launch_choice(prec):
    """Chunks 1, 2, 3, 8 (more chunks than a polynomial has monomials), both
    launch shapes, partial-tile groups capped at 1 or 16: every output within
    the tolerance of the exact oracle; then the autotuner's choice."""
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, points = _small_batch(prec)
    code = pe_precision(prec)
    many = pkg.PolyEvalMany([s.as_fp64() if prec == "f64" else s for s in systems], [x.shape[1] for x in points],
                            code)
    pb, fb, Jb = many.buffers()
    many.pack_points([_device_points(prec, x) for x in points], pb)
    for groups in (1, 16):
        for chunks in (1, 2, 3, 8):
            for shape in (1, 2):
                many.set_launch(chunks, shape, groups)
                fb.fill_(np.nan)
                Jb.fill_(np.nan)
                many.eval_buffers(pb, fb, Jb)
                torch.cuda.synchronize()
                assert pkg.polyeval_status(many.handle) == pkg.PE_OK
                fs, Js = many.views(fb, Jb)
                _check_batch(prec, systems, points, fs, Js)
    chunks, shape, groups = many.autotune(pb, fb, Jb)
    assert chunks in (1, 2, 4, 8) and shape in (1, 2)
    assert groups in ((1,) if prec in ("ddint", "qd") else (1, 16))
    fb.fill_(np.nan)
    Jb.fill_(np.nan)
    many.eval_buffers(pb, fb, Jb)
    torch.cuda.synchronize()
    fs, Js = many.views(fb, Jb)
    _check_batch(prec, systems, points, fs, Js)
    with pytest.raises(pkg.PolyEvalError):
        pkg.polyeval_autotune(many.handle, pb, 5, fb, Jb)
    with pytest.raises(pkg.PolyEvalError):
        pkg.polyeval_set_launch(many.handle, 3, 1, 1, 1)


@pytest.mark.parametrize("prec", ["dd", "ddint"])
def test_config4_autotuned_batch(prec):
    """The 200-system workload after polyeval_autotune: the six smallest
    systems in full against the C double-double oracle, five sampled systems
    against the exact oracle at one output row each."""
    import torch

    import oracle
    import paper_1201_0499_gb300 as pkg

    systems, pts = synth.config(4)
    many = pkg.PolyEvalMany(systems, [p.shape[1] for p in pts], pe_precision(prec))
    pb, fb, Jb = many.buffers()
    many.pack_points([to_device(p) for p in pts], pb)
    chunks, shape, groups = many.autotune(pb, fb, Jb)
    assert chunks >= 1 and shape in (1, 2) and groups in (1, 16)
    fb.zero_()
    Jb.zero_()
    many.eval_buffers(pb, fb, Jb)
    torch.cuda.synchronize()
    assert pkg.polyeval_status(many.handle) == pkg.PE_OK
    fs, Js = many.views(fb, Jb)
    order = np.argsort([s.n_monos * p.shape[1] for s, p in zip(systems, pts)])
    for si in order[:6]:
        s, x = systems[si], pts[si]
        f, J = fs[si].cpu().numpy(), Js[si].cpu().numpy()
        Fo, Jo = oracle.dd_eval(s, x, threads=0)
        Sf, SJ = scales(s, x)
        assert normwise_vs(f, Fo, Sf) <= DD_TOL, si
        assert normwise_vs(J, Jo, SJ) <= DD_TOL, si
    rng = np.random.Generator(np.random.PCG64(631))
    for si in rng.choice(len(systems), size=5, replace=False):
        s, x = systems[si], pts[si]
        q = int(rng.integers(0, x.shape[1]))
        p = int(rng.integers(0, s.n_polys))
        ef, ej = E.max_errors(s, x, fs[si].cpu().numpy(), Js[si].cpu().numpy(), [q], polys=[p])
        assert ef <= DD_TOL and ej <= DD_TOL, (si, ef, ej)


@pytest.mark.parametrize("prec", ["dd", "qd"])
def test_batch_cuda_graph_replay_matches_eager(prec):
    """A batch evaluation (power table, chunked monomial kernel, combine or
    quad-double finalize) captured in a CUDA graph and replayed gives the same
    bits as the eager call."""
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, points = _small_batch(prec)
    many = pkg.PolyEvalMany(systems, [x.shape[1] for x in points], pe_precision(prec))
    pb, fb, Jb = many.buffers()
    many.pack_points([_device_points(prec, x) for x in points], pb)
    many.set_launch(3, 2, 16)
    many.eval_buffers(pb, fb, Jb)
    torch.cuda.synchronize()
    f_ref, J_ref = fb.clone(), Jb.clone()
    g = torch.cuda.CUDAGraph()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        many.eval_buffers(pb, fb, Jb)  # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(side)
    with torch.cuda.graph(g):
        many.eval_buffers(pb, fb, Jb)
    fb.zero_()
    Jb.zero_()
    g.replay()
    torch.cuda.synchronize()
    assert pkg.polyeval_status(many.handle) == pkg.PE_OK
    assert torch.equal(fb, f_ref) and torch.equal(Jb, J_ref)


def test_batch_without_points_autotunes_and_evaluates():
    """A batch whose systems all have no points: evaluation is a no-op and the
    autotuner reports the launch in place."""
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, _ = _small_batch("dd")
    many = pkg.PolyEvalMany(systems[:3], [0, 0, 0], pkg.PE_DD)
    x = torch.zeros(2, 4, dtype=torch.float64, device="cuda")
    chunks, shape, groups = pkg.polyeval_autotune(many.handle, x, 0, x, x)
    assert chunks >= 1 and shape in (1, 2) and groups in (1, 16)
    pkg.polyeval_eval_many(many.handle, x, x, x)
    torch.cuda.synchronize()
    assert pkg.polyeval_status(many.handle) == pkg.PE_OK


@pytest.fixture(scope="module")
def config4_rows():
    """The 200-system workload with one seeded point per system (every
    system has at least one point): the C double-double oracle's outputs at
    that point on the double-double inputs and on the inputs rounded to
    double, and the normwise scales."""
    import concurrent.futures as cf
    import os

    import oracle

    systems, pts = synth.config(4)
    rng = np.random.Generator(np.random.PCG64(641))
    qs = [int(rng.integers(0, x.shape[1])) for x in pts]

    def one(args):  # one point per call: the systems run side by side on the host cores
        s, x, q = args
        sub = np.ascontiguousarray(x[:, q:q + 1])
        s64, p64 = fp64_inputs(s, sub)
        return q, oracle.dd_eval(s, sub, threads=1), oracle.dd_eval(s64, p64, threads=1), scales(s, sub)

    with cf.ThreadPoolExecutor(max_workers=os.cpu_count() or 4) as ex:
        rows = list(ex.map(one, zip(systems, pts, qs)))
    return systems, pts, rows


@pytest.mark.parametrize("prec", ["dd", "ddint", "f64"])
def test_config4_every_system_at_a_seeded_point(prec, config4_rows):
    """Every one of the 200 systems, at one seeded point each, every output
    (all polynomials, every J entry) against the C double-double oracle,
    after the batch autotuner picked the launch."""
    import torch

    import paper_1201_0499_gb300 as pkg

    systems, pts, rows = config4_rows
    dd = prec != "f64"
    many = pkg.PolyEvalMany([s if dd else s.as_fp64() for s in systems], [p.shape[1] for p in pts],
                            pe_precision(prec))
    pb, fb, Jb = many.buffers()
    many.pack_points([to_device(p, dd) for p in pts], pb)
    many.autotune(pb, fb, Jb)
    many.eval_buffers(pb, fb, Jb)
    torch.cuda.synchronize()
    assert pkg.polyeval_status(many.handle) == pkg.PE_OK
    fs, Js = many.views(fb, Jb)
    for si, (q, ref_dd, ref_64, (Sf, SJ)) in enumerate(rows):
        f = fs[si][:, q:q + 1].cpu().numpy()
        J = Js[si][:, :, q:q + 1].cpu().numpy()
        Fo, Jo = ref_dd if dd else ref_64
        if not dd:
            f, J = widen(f), widen(J)
        assert normwise_vs(f, Fo, Sf) <= tol(prec), si
        assert normwise_vs(J, Jo, SJ) <= tol(prec), si
    many.close()


def test_config4_quad_double_every_system_one_row():
    """Quad-double on the 200-system batch: for every system one row (one
    polynomial, all of its J entries) at a seeded point against the exact
    oracle at 1e-60."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import QD_TOL

    systems, pts = synth.config(4)
    rng = np.random.Generator(np.random.PCG64(651))
    qs = [s.to_qd(652 + i) for i, s in enumerate(systems)]
    qp = [synth.widen_qd(rng, p) for p in pts]
    picks = [(int(rng.integers(0, p.shape[1])), int(rng.integers(0, s.n_polys))) for s, p in zip(qs, qp)]
    jobs = [(s, np.ascontiguousarray(p[:, q:q + 1]), 0, [poly]) for s, p, (q, poly) in zip(qs, qp, picks)]
    with cf.ProcessPoolExecutor(max_workers=16, mp_context=mp.get_context("spawn")) as ex:
        exact = list(ex.map(E.evaluate_point, *zip(*jobs)))
    many = pkg.PolyEvalMany(qs, [p.shape[1] for p in qp], pkg.PE_QD_INT)
    pb, fb, Jb = many.buffers()
    many.pack_points([to_device(p) for p in qp], pb)
    many.eval_buffers(pb, fb, Jb)
    torch.cuda.synchronize()
    assert pkg.polyeval_status(many.handle) == pkg.PE_OK
    fs, Js = many.views(fb, Jb)
    for si, ((q, poly), (f, J), job) in enumerate(zip(picks, exact, jobs)):
        Sf, SJ = E.scales_point(job[0], job[1], 0, polys=[poly])
        assert E.normwise_error(fs[si][poly, q].cpu().numpy(), f[poly], Sf[poly]) <= QD_TOL, si
        Jrow = Js[si][poly, :, q].cpu().numpy()
        ej = max(E.normwise_error(Jrow[i], J[poly].get(i, E.ZERO), SJ[poly].get(i, 0.0))
                 for i in range(qs[si].n_vars))
        assert ej <= QD_TOL, (si, ej)
    many.close()
