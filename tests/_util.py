"""Helpers shared by the tests: running the CUDA path and measuring errors.

Error measure (the one the accuracy targets are stated in): for an output z
with exact value z*, |z - z*| / S where S is the same sum over absolute
values (S_f = sum |c| |x^a|, S_J = sum |c| a_i |x^(a-e_i)|).  Outputs whose S
is zero must be exactly zero.
"""
from __future__ import annotations

import numpy as np

DD_TOL = 1e-28
F64_TOL = 1e-13
# quad-double: products err by about 2^-246, each sum by 2^-219 of its largest
# term, the final rounding by 2^-211 of the value; 1e-60 leaves a factor of
# several hundred over that bound (and is 1e32 times tighter than DD_TOL)
QD_TOL = 1e-60

# the precisions of the library: double-double, double, double-double with
# integer-pipe products
PRECS = ["dd", "f64", "ddint"]


def tol(prec):
    return F64_TOL if prec == "f64" else QD_TOL if prec == "qd" else DD_TOL


def pe_precision(prec):
    import paper_1201_0499_gb300 as pkg

    return {"dd": pkg.PE_DD, "f64": pkg.PE_F64, "ddint": pkg.PE_DD_INT, "qd": pkg.PE_QD_INT}[prec]


def widen(x2):
    """[..., 2] complex doubles -> [..., 4] complex double-doubles with zero low words."""
    out = np.zeros(x2.shape[:-1] + (4,))
    out[..., 0] = x2[..., 0]
    out[..., 2] = x2[..., 1]
    return out


def fp64_inputs(system, pts):
    """The inputs of the complex-double path, as double-doubles with zero low words."""
    p = pts.copy()
    p[..., 1] = 0.0
    p[..., 3] = 0.0
    return system.as_fp64(), p


def to_device(pts, dd=True):
    import torch

    a = pts if dd else np.ascontiguousarray(pts[..., [0, 2]])
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def run(system, pts, prec="dd", max_points=None):
    """Evaluate with the CUDA library; returns numpy f [N,P,4], J [N,n,P,4].
    prec: "dd", "f64" or "ddint" (True/False stand for "dd"/"f64")."""
    import torch

    import paper_1201_0499_gb300 as pkg

    if prec is True:
        prec = "dd"
    elif prec is False:
        prec = "f64"
    dd = prec != "f64"
    P = pts.shape[1]
    ev = pkg.PolyEval(system if dd else system.as_fp64(), pe_precision(prec),
                      max_points=max(P, 1) if max_points is None else max_points)
    f, J = ev.eval(to_device(pts, dd))
    torch.cuda.synchronize()
    assert ev.status() == pkg.PE_OK
    f, J = f.cpu().numpy(), J.cpu().numpy()
    ev.close()
    if not dd:
        f, J = widen(f), widen(J)
    return f, J


def scales(system, pts):
    """Normwise scales for all points: S_f [N, P], S_J [N, n, P] (float64).

    Vectorised over monomials; the product over all variables but one is
    taken from exclusive prefix and suffix products, so zero coordinates are
    handled exactly."""
    n, N, P = system.n_vars, system.n_polys, pts.shape[1]
    M = system.n_monos
    Sf = np.zeros((N, P))
    SJ = np.zeros((N, n, P))
    if M == 0:
        return Sf, SJ
    k = np.diff(system.mono_ptr).astype(np.int64)
    kmax = int(k.max()) if k.size else 0
    poly_of = np.repeat(np.arange(N), np.diff(system.poly_ptr))
    ac = np.hypot(system.coef[:, 0], system.coef[:, system.coef.shape[1] // 2])
    rows = np.repeat(np.arange(M), k)
    cols = np.arange(system.pos.size) - np.repeat(system.mono_ptr[:-1], k)
    ax_all = np.hypot(pts[..., 0], pts[..., pts.shape[-1] // 2])  # [n, P]
    for q in range(P):
        ax = ax_all[:, q]
        W = np.ones((M, max(kmax, 1)))
        Wd = np.ones((M, max(kmax, 1)))
        W[rows, cols] = ax[system.pos] ** system.exp
        Wd[rows, cols] = system.exp * ax[system.pos] ** (system.exp - 1)
        pre = np.cumprod(np.concatenate([np.ones((M, 1)), W[:, :-1]], axis=1), axis=1)
        suf = np.cumprod(np.concatenate([np.ones((M, 1)), W[:, :0:-1]], axis=1), axis=1)[:, ::-1]
        full = pre[:, -1] * W[:, -1]
        np.add.at(Sf[:, q], poly_of, ac * full)
        d = ac[rows] * Wd[rows, cols] * pre[rows, cols] * suf[rows, cols]
        np.add.at(SJ[:, :, q], (poly_of[rows], system.pos), d)
    return Sf, SJ


def dd_diff(a, b):
    """|a - b| for complex multi-double arrays [..., 4] or [..., 8] (the
    parts of each component subtracted pairwise), in float64."""
    w = a.shape[-1] // 2
    re = sum(a[..., i] - b[..., i] for i in range(w))
    im = sum(a[..., w + i] - b[..., w + i] for i in range(w))
    return np.hypot(re, im)


def normwise_vs(a, b, S):
    """Largest |a - b| / S; entries with S == 0 must agree exactly (inf if not)."""
    d = dd_diff(a, b)
    zero = S == 0
    if np.any(zero):
        if not (np.all(a[zero] == 0.0) and np.all(b[zero] == 0.0)):
            return np.inf
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(zero, 0.0, d / np.where(zero, 1.0, S))
    return float(np.max(r)) if r.size else 0.0


def square_system(seed, n, m, kmax, emax):
    """A square system of n polynomials in n variables: a constant term (which
    keeps the Jacobian generic) and m random monomials each."""
    import synth

    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for _p in range(n):
        mons = [([], [])]
        for _t in range(m):
            k = int(rng.integers(1, kmax + 1))
            pos = sorted(rng.choice(n, size=k, replace=False).tolist())
            mons.append((pos, rng.integers(1, emax + 1, size=k).tolist()))
        polys.append(mons)
    return synth.from_monomials(n, polys, synth.random_cdd(rng, n * (m + 1)))


def fr_parts(v):
    """A complex double-double [4] or quad-double [8] as an exact pair of
    Fractions (re, im)."""
    from fractions import Fraction

    w = len(v) // 2
    return (sum((Fraction(float(a)) for a in v[:w]), Fraction(0)),
            sum((Fraction(float(a)) for a in v[w:]), Fraction(0)))


def cabs(z):
    return abs(complex(float(z[0]), float(z[1])))
