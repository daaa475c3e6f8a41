"""The two large single-system workloads at full size, in the launch the
benchmark times, sampled densely: n = 64 (m = 256, k = 16, 4096 points) and
n = 128 (m = 1024, k = 32, 16384 points).

At each workload the GPU evaluates the whole batch; then every output (all
polynomials, every Jacobian entry) of the first and the last tile of 16
points and of 16 seeded points between them is compared with the C
double-double oracle (itself within 1e-30 of exact), for double-double on the
FP64 pipe, double-double with integer-pipe products, and complex double (on
the inputs rounded to double, against the oracle run on those).  A few of
those outputs are also checked against the exact oracle (Section 2, Eq. 1).
Oracle values are computed once per workload; the exact ones in a spawned
process pool.
"""
import concurrent.futures as cf
import multiprocessing as mp

import numpy as np
import pytest

import synth
from oracle import exact as E

from _util import fp64_inputs, normwise_vs, pe_precision, scales, tol

pytestmark = pytest.mark.gpu

TILE = 16


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1201_0499_gb300 as pkg

    pkg.load_library()
    torch.cuda.set_device(0)


def sample_points(P, seed):
    """The first and last tile and 16 seeded points in between, in order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mid = sorted(rng.choice(np.arange(TILE, P - TILE), size=16, replace=False).tolist())
    return list(range(TILE)) + mid + list(range(P - TILE, P))


def _reference(cfg, seed, exact_pairs):
    import oracle

    s, pts = synth.config(cfg)
    idx = sample_points(pts.shape[1], seed)
    assert len(set(idx)) == 3 * TILE and idx[-1] == pts.shape[1] - 1
    sub = np.ascontiguousarray(pts[:, idx])
    s64, p64 = fp64_inputs(s, sub)
    ref = {"system": s, "pts": pts, "idx": idx, "sub": sub, "sub64": p64, "system64": s64}
    ref["dd"] = oracle.dd_eval(s, sub, threads=0)
    ref["f64"] = oracle.dd_eval(s64, p64, threads=0)
    ref["scales"] = scales(s, sub)
    # exact values: (column of the sample, polynomial) pairs, dd inputs and double inputs
    jobs = [(s, sub, c, [p]) for c, p in exact_pairs] + [(s64, p64, c, [p]) for c, p in exact_pairs[:2]]
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(E.evaluate_point, *zip(*jobs)))
    out = []
    for (sy, pt, c, (p,)), (f, J) in zip(jobs, res):
        Sf, SJ = E.scales_point(sy, pt, c, polys=[p])
        out.append(((c, p), (f[p], J[p], Sf[p], SJ[p])))
    ref["exact_dd"], ref["exact_f64"] = out[:len(exact_pairs)], out[len(exact_pairs):]
    return ref


@pytest.fixture(scope="module")
def ref3():
    return _reference(3, 331, [(0, 0), (20, 17), (47, 63), (31, 40)])


@pytest.fixture(scope="module")
def ref5():
    return _reference(5, 551, [(0, 0), (47, 127), (24, 64), (15, 3)])


def _gpu_sampled(prec, ref):
    """Evaluate the whole batch in `prec`; return the sampled outputs as
    complex double-double arrays f [N, S, 4], J [N, n, S, 4]."""
    import torch

    import paper_1201_0499_gb300 as pkg

    s, pts = ref["system"], ref["pts"]
    P = pts.shape[1]
    dd = prec != "f64"
    x = torch.from_numpy(np.ascontiguousarray(pts if dd else pts[..., [0, 2]])).cuda()
    ev = pkg.PolyEval(s if dd else s.as_fp64(), pe_precision(prec), max_points=P)
    f, J = ev.eval(x)
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    idx = torch.tensor(ref["idx"], device="cuda")
    fs = f.index_select(1, idx).cpu().numpy()
    Js = J.index_select(2, idx).cpu().numpy()
    ev.close()
    del f, J, x
    torch.cuda.empty_cache()
    if not dd:
        w = np.zeros(fs.shape[:-1] + (4,))
        w[..., 0], w[..., 2] = fs[..., 0], fs[..., 1]
        fs = w
        w = np.zeros(Js.shape[:-1] + (4,))
        w[..., 0], w[..., 2] = Js[..., 0], Js[..., 1]
        Js = w
    return fs, Js


def _check(prec, ref):
    fs, Js = _gpu_sampled(prec, ref)
    Fo, Jo = ref["f64" if prec == "f64" else "dd"]
    Sf, SJ = ref["scales"]
    assert normwise_vs(fs, Fo, Sf) <= tol(prec)
    assert normwise_vs(Js, Jo, SJ) <= tol(prec)
    n = ref["system"].n_vars
    for (c, p), (fx, Jx, sf, sj) in ref["exact_f64" if prec == "f64" else "exact_dd"]:
        assert E.normwise_error(fs[p, c], fx, sf) <= tol(prec), (c, p)
        ej = max(E.normwise_error(Js[p, i, c], Jx.get(i, E.ZERO), sj.get(i, 0.0)) for i in range(n))
        assert ej <= tol(prec), (c, p, ej)


@pytest.mark.parametrize("prec", ["dd", "ddint", "f64"])
def test_n64_dense_samples(prec, ref3):
    _check(prec, ref3)


@pytest.mark.parametrize("prec", ["dd", "ddint", "f64"])
def test_n128_dense_samples(prec, ref5):
    _check(prec, ref5)



def _qd_reference(cfg, seed, pairs):
    """Quad-double data of the workload (the double-double values with two
    random lower parts) and exact rows at (point, polynomial) pairs."""
    s, pts = synth.config(cfg)
    rng = np.random.Generator(np.random.PCG64(seed))
    sq, pq = s.to_qd(seed + 1), synth.widen_qd(rng, pts)
    cols = sorted({q for q, _ in pairs})
    sub = np.ascontiguousarray(pq[:, cols])
    jobs = [(sq, sub, cols.index(q), [p]) for q, p in pairs]
    with cf.ProcessPoolExecutor(max_workers=len(jobs), mp_context=mp.get_context("spawn")) as ex:
        res = list(ex.map(E.evaluate_point, *zip(*jobs)))
    rows = []
    for (sy, pt, c, (p,)), (f, J) in zip(jobs, res):
        Sf, SJ = E.scales_point(sy, pt, c, polys=[p])
        rows.append((pairs[len(rows)], (f[p], J[p], Sf[p], SJ[p])))
    return {"system": sq, "pts": pq, "rows": rows}


def _check_qd_rows(ref):
    import torch

    import paper_1201_0499_gb300 as pkg
    from _util import QD_TOL

    s, pts = ref["system"], ref["pts"]
    P = pts.shape[1]
    ev = pkg.PolyEval(s, pkg.PE_QD_INT, max_points=P)
    f, J = ev.eval(torch.from_numpy(pts).cuda())
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    for (q, p), (fx, Jx, sf, sj) in ref["rows"]:
        fq = f[p, q].cpu().numpy()
        Jq = J[p, :, q].cpu().numpy()
        assert E.normwise_error(fq, fx, sf) <= QD_TOL, (q, p)
        ej = max(E.normwise_error(Jq[i], Jx.get(i, E.ZERO), sj.get(i, 0.0)) for i in range(s.n_vars))
        assert ej <= QD_TOL, (q, p, ej)
    ev.close()


def test_n64_quad_double_rows():
    """Quad-double on the whole n = 64 batch (4096 points): rows at both ends
    and in between against the exact oracle at 1e-60."""
    _check_qd_rows(_qd_reference(3, 333, [(0, 0), (15, 63), (2047, 31), (4080, 7), (4095, 63), (4095, 0)]))


def test_n128_quad_double_rows():
    """Quad-double on the whole n = 128 batch (16384 points): rows at both
    ends and in between against the exact oracle at 1e-60."""
    _check_qd_rows(_qd_reference(5, 555, [(0, 0), (15, 127), (8191, 64), (16368, 5), (16383, 127), (16383, 0)]))
