"""Seeded synthetic polynomial systems and evaluation points.

This module only draws inputs.  It holds none of the evaluation arithmetic:
both the oracle (``oracle/``) and the CUDA path (``paper_1201_0499_gb300``)
read the plain arrays it returns.

Problem format (Section 2, Eq. 1 of Verschelde & Yoffe): a polynomial is a
tuple (C, A) of nonzero complex coefficients and exponent vectors; a system is
a tuple of such polynomials.  The regular benchmark family of Section 2 fixes
the number k of variables per monomial, a maximal degree d per variable and the
number m of monomials per polynomial.  Monomials are sparse: positions
i_1 < ... < i_k with exponents a >= 1.

Arrays (CSR by polynomial, then by monomial):

* ``poly_ptr``  int64 [N+1]  monomial offsets of each polynomial
* ``mono_ptr``  int64 [M+1]  offsets of each monomial into ``pos``/``exp``
* ``pos``       int32 [nnz]  0-based variable index, strictly increasing
                             inside a monomial
* ``exp``       int32 [nnz]  exponent >= 1
* ``coef``      float64 [M, 4]  complex double-double (re_hi, re_lo,
                                im_hi, im_lo), or [M, 8] complex
                                quad-double (re0..re3, im0..im3)

Points are float64 [n, P, 4]: structure of arrays, variable-major, each entry
a complex double-double ([n, P, 8] for quad-double points).

Every random draw goes through numpy's PCG64 and only IEEE basic operations
(+, -, *, /, exact scaling by powers of two), so the same seed gives the same
bits on x86-64 and on AArch64.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

SEED_BASE = 12010499


@dataclass
class System:
    n_vars: int
    n_polys: int
    poly_ptr: np.ndarray
    mono_ptr: np.ndarray
    pos: np.ndarray
    exp: np.ndarray
    coef: np.ndarray
    meta: dict = field(default_factory=dict)

    @property
    def n_monos(self) -> int:
        return int(self.poly_ptr[-1])

    @property
    def max_exp(self) -> int:
        return int(self.exp.max()) if self.exp.size else 1

    def monomial(self, t: int):
        """(positions, exponents) of monomial t as Python lists."""
        a, b = int(self.mono_ptr[t]), int(self.mono_ptr[t + 1])
        return self.pos[a:b].tolist(), self.exp[a:b].tolist()

    def as_fp64(self) -> "System":
        """Same system with every coefficient part but the leading one of
        each component set to zero."""
        w = self.coef.shape[1] // 2
        c = np.zeros_like(self.coef)
        c[:, 0] = self.coef[:, 0]
        c[:, w] = self.coef[:, w]
        return System(self.n_vars, self.n_polys, self.poly_ptr, self.mono_ptr, self.pos, self.exp, c, dict(self.meta))

    def to_qd(self, seed: int) -> "System":
        """Same monomials, coefficients widened to quad-double: the
        double-double parts kept and two random lower parts added
        (``widen_qd``)."""
        rng = np.random.Generator(np.random.PCG64(seed))
        return System(self.n_vars, self.n_polys, self.poly_ptr, self.mono_ptr, self.pos, self.exp,
                      widen_qd(rng, self.coef), dict(self.meta))


# ----------------------------------------------------------------------------
# random double-double numbers
# ----------------------------------------------------------------------------

def _u53(rng, size):
    """Uniform doubles in [0, 1) with 53 random bits."""
    return rng.integers(0, 1 << 53, size=size, dtype=np.int64).astype(np.float64) * (2.0 ** -53)


def _low_words(rng, hi):
    """Random low words with |lo| < ulp(hi)/4, so (hi, lo) stays normalised."""
    hi = np.asarray(hi, dtype=np.float64)
    _, e = np.frexp(hi)  # hi = m * 2**e, 0.5 <= |m| < 1, ulp(hi) = 2**(e-53)
    j = rng.integers(0, 1 << 52, size=hi.shape, dtype=np.int64) - (1 << 51)
    lo = np.ldexp(j.astype(np.float64), (e - 106).astype(np.int32))
    lo[hi == 0.0] = 0.0
    return lo


def _unit_circle(rng, size):
    """Points near the unit circle: rational parametrisation, then a random
    quarter turn; (1-t^2)/(1+t^2) and 2t/(1+t^2) use only IEEE basic ops."""
    t = 2.0 * _u53(rng, size) - 1.0
    den = 1.0 + t * t
    re = (1.0 - t * t) / den
    im = (2.0 * t) / den
    q = rng.integers(0, 4, size=size)
    re2 = np.where(q == 0, re, np.where(q == 1, -im, np.where(q == 2, -re, im)))
    im2 = np.where(q == 0, im, np.where(q == 1, re, np.where(q == 2, -im, -re)))
    return re2, im2


def _log_uniform_by_octave(rng, size, e_lo, e_hi):
    """Moduli m * 2**e with e uniform in [e_lo, e_hi] and m uniform in [1, 2)."""
    m = 1.0 + _u53(rng, size)
    e = rng.integers(e_lo, e_hi + 1, size=size)
    return np.ldexp(m, e.astype(np.int32))


def random_cdd(rng, size, modulus=None):
    """Complex double-doubles near the unit circle, optionally scaled by
    ``modulus`` (an array of the same size).  Returns float64 [size, 4]."""
    re, im = _unit_circle(rng, size)
    if modulus is not None:
        re = re * modulus
        im = im * modulus
    out = np.empty((size, 4), dtype=np.float64)
    out[:, 0] = re
    out[:, 1] = _low_words(rng, re)
    out[:, 2] = im
    out[:, 3] = _low_words(rng, im)
    return out


def widen_qd(rng, cdd):
    """Complex double-doubles [..., 4] to complex quad-doubles [..., 8]: the
    two parts of each component kept, then two random lower parts, each below
    a quarter unit in the last place of the part before it (so the result is
    a normalised quad-double when the input is a normalised double-double)."""
    cdd = np.asarray(cdd, dtype=np.float64)
    out = np.empty(cdd.shape[:-1] + (8,), dtype=np.float64)
    for c in range(2):
        out[..., 4 * c] = cdd[..., 2 * c]
        out[..., 4 * c + 1] = cdd[..., 2 * c + 1]
        out[..., 4 * c + 2] = _low_words(rng, out[..., 4 * c + 1])
        out[..., 4 * c + 3] = _low_words(rng, out[..., 4 * c + 2])
    return out


# ----------------------------------------------------------------------------
# systems
# ----------------------------------------------------------------------------

def _draw_rows(rng, need, n, k, e_min, e_max, kmax):
    """``need`` monomials as padded rows: positions (sorted, padded with n),
    exponents (padded with 0).  ``k`` is an int array of per-row sizes."""
    keys = rng.random((need, n))
    perm = np.argsort(keys, axis=1)  # a uniform random permutation per row
    chosen = np.arange(n)[None, :] < k[:, None]
    S = np.sort(np.where(chosen, perm, n), axis=1)[:, :kmax].astype(np.int32)
    A = rng.integers(e_min, e_max + 1, size=(need, kmax)).astype(np.int32)
    A[np.arange(kmax)[None, :] >= k[:, None]] = 0
    return S, A


def _homogenise(rng, k, degree, e_max, need):
    """Exponent rows that start at 1 and receive (degree - k) units, each on a
    uniformly chosen position whose exponent is still below e_max."""
    extra = degree - k
    if extra < 0 or extra > k * (e_max - 1):
        raise ValueError("homogeneous degree out of reach")
    A = np.ones((need, k), dtype=np.int32)
    for _u in range(extra):
        open_ = A < e_max
        cnt = open_.sum(axis=1)
        pick = np.floor(_u53(rng, need) * cnt).astype(np.int64)  # 0 <= pick < cnt
        rank = np.cumsum(open_, axis=1) - 1
        hit = open_ & (rank == pick[:, None])
        A += hit.astype(np.int32)
    return A


def _unique_in_order(S, A):
    """Indices of the first occurrence of each distinct (positions, exponents)
    row, in their original order."""
    rows = np.concatenate([S, A], axis=1)
    _, first = np.unique(rows, axis=0, return_index=True)
    return np.sort(first)


def _poly(rng, n, m, k_of, e_min, e_max, kmax, homogeneous_degree=None):
    """One polynomial of m distinct monomials (duplicates are drawn again)."""
    S = np.zeros((0, kmax), dtype=np.int32)
    A = np.zeros((0, kmax), dtype=np.int32)
    K = np.zeros(0, dtype=np.int64)
    while S.shape[0] < m:
        need = m - S.shape[0]
        k = k_of(need)
        s, a = _draw_rows(rng, need, n, k, e_min, e_max, kmax)
        if homogeneous_degree is not None:
            a = _homogenise(rng, kmax, homogeneous_degree, e_max, need)
        S, A, K = np.concatenate([S, s]), np.concatenate([A, a]), np.concatenate([K, k])
        keep = _unique_in_order(S, A)
        S, A, K = S[keep], A[keep], K[keep]
    return S[:m], A[:m], K[:m]


def _assemble(n, polys, coef, meta):
    """polys: list of (S, A, K) padded rows per polynomial."""
    kmax = max((p[0].shape[1] for p in polys), default=0)
    counts = np.asarray([p[0].shape[0] for p in polys], dtype=np.int64)
    K = np.concatenate([p[2] for p in polys]) if polys else np.zeros(0, np.int64)
    pos_parts, exp_parts = [], []
    for S, A, k in polys:
        mask = np.arange(S.shape[1])[None, :] < k[:, None]
        pos_parts.append(S[mask])
        exp_parts.append(A[mask])
    poly_ptr = np.concatenate([[0], np.cumsum(counts)]).astype(np.int64)
    mono_ptr = np.concatenate([[0], np.cumsum(K)]).astype(np.int64)
    return System(
        n_vars=n,
        n_polys=len(polys),
        poly_ptr=poly_ptr,
        mono_ptr=mono_ptr,
        pos=np.concatenate(pos_parts).astype(np.int32) if pos_parts else np.zeros(0, np.int32),
        exp=np.concatenate(exp_parts).astype(np.int32) if exp_parts else np.zeros(0, np.int32),
        coef=np.ascontiguousarray(coef, dtype=np.float64),
        meta=dict(meta, kmax=kmax),
    )


def regular_system(seed, n, m, k, e_max, e_min=1, n_polys=None, coef_modulus=None, homogeneous_degree=None):
    """The regular family of Section 2: every polynomial has m monomials, every
    monomial k distinct variables, exponents uniform in [e_min, e_max].

    ``coef_modulus``: None for unit-circle coefficients, or (e_lo, e_hi) for
    moduli log-uniform by octave in [2**e_lo, 2**(e_hi+1)).
    ``homogeneous_degree``: if set, every monomial starts with all exponents 1
    and receives (degree - k) extra units, each on a uniformly chosen position
    whose exponent is still below e_max."""
    rng = np.random.Generator(np.random.PCG64(seed))
    N = n if n_polys is None else n_polys
    polys = [_poly(rng, n, m, lambda c: np.full(c, k, dtype=np.int64), e_min, e_max, k, homogeneous_degree)
             for _p in range(N)]
    M = N * m
    mod = None
    if coef_modulus is not None:
        mod = _log_uniform_by_octave(rng, M, coef_modulus[0], coef_modulus[1])
    coef = random_cdd(rng, M, mod)
    meta = dict(seed=seed, n=n, m=m, k=k, e_min=e_min, e_max=e_max, coef_modulus=coef_modulus,
                homogeneous_degree=homogeneous_degree)
    return _assemble(n, polys, coef, meta)


def ragged_systems(seed, count=200, n_range=(8, 128), m_range=(8, 512), k_max=24, e_max=6, p_range=(1, 256)):
    """Many systems of uneven shape: n uniform per system, m uniform per
    polynomial, k uniform in [2, min(n, k_max)] per monomial, exponents in
    [1, e_max], unit-circle coefficients; and a point count per system."""
    rng = np.random.Generator(np.random.PCG64(seed))
    systems, npts = [], []
    for s in range(count):
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        kmax = min(n, k_max)
        polys = []
        for _p in range(n):
            m = int(rng.integers(m_range[0], m_range[1] + 1))
            polys.append(_poly(rng, n, m, lambda c: rng.integers(2, kmax + 1, size=c).astype(np.int64),
                               1, e_max, kmax))
        total = sum(p[0].shape[0] for p in polys)
        coef = random_cdd(rng, total)
        systems.append(_assemble(n, polys, coef, dict(seed=seed, index=s, n=n, e_max=e_max)))
        npts.append(int(rng.integers(p_range[0], p_range[1] + 1)))
    return systems, npts


def points(seed, n, P, modulus_octaves=None):
    """P evaluation points, float64 [n, P, 4].  ``modulus_octaves``: None for
    the unit circle, or (e_lo, e_hi) for |x| log-uniform by octave."""
    rng = np.random.Generator(np.random.PCG64(seed))
    size = n * P
    mod = None
    if modulus_octaves is not None:
        mod = _log_uniform_by_octave(rng, size, modulus_octaves[0], modulus_octaves[1])
    return random_cdd(rng, size, mod).reshape(n, P, 4)


# ----------------------------------------------------------------------------
# the five workloads (seeds SEED_BASE + config number)
# ----------------------------------------------------------------------------

CONFIG_TEXT = {
    1: "tiny: n=16, 16 polynomials, m=8, k=4, exponents 1..3, unit-circle coefficients, 1 point",
    2: "n=32, 32 polynomials, m=64, k=9, exponents 1..5, unit-circle coefficients and points, 1024 points",
    3: "n=64, 64 polynomials, m=256, k=16, exponents 1..8, |c| log-uniform 2^-10..2^10, 4096 points |x| in [0.5,2)",
    4: "ragged: 200 systems, n in [8,128], m in [8,512] per polynomial, k in [2,min(n,24)], exponents 1..6, 1..256 points each",
    5: "large: n=128, 128 polynomials, m=1024, k=32, exponents 1..4, unit-circle coefficients, 16384 points",
}


def config(i: int, homogeneous: bool = False, n_points: Optional[int] = None):
    """Return (system, points) for configs 1, 2, 3, 5; for config 4 return
    (list of systems, list of point arrays)."""
    seed = SEED_BASE + i
    if i == 1:
        s = regular_system(seed, 16, 8, 4, 3)
        return s, points(seed + 1000, 16, 1 if n_points is None else n_points)
    if i == 2:
        s = regular_system(seed, 32, 64, 9, 5)
        return s, points(seed + 1000, 32, 1024 if n_points is None else n_points)
    if i == 3:
        if homogeneous:
            s = regular_system(seed + 500, 64, 256, 16, 8, coef_modulus=(-10, 9), homogeneous_degree=24)
        else:
            s = regular_system(seed, 64, 256, 16, 8, coef_modulus=(-10, 9))
        return s, points(seed + 1000, 64, 4096 if n_points is None else n_points, modulus_octaves=(-1, 0))
    if i == 4:
        systems, npts = ragged_systems(seed)
        pts = [points(seed + 1000 + j, s.n_vars, npts[j] if n_points is None else min(npts[j], n_points))
               for j, s in enumerate(systems)]
        return systems, pts
    if i == 5:
        s = regular_system(seed, 128, 1024, 32, 4)
        return s, points(seed + 1000, 128, 16384 if n_points is None else n_points)
    raise ValueError(f"no config {i}")


def from_monomials(n, polys, coef):
    """A system from explicit monomials: ``polys`` is a list (per polynomial)
    of lists of (positions, exponents); ``coef`` is float64 [M, 4] in the same
    order.  Positions must be strictly increasing inside a monomial."""
    rows = []
    for mons in polys:
        kmax = max((len(p) for p, _ in mons), default=0)
        S = np.full((len(mons), kmax), n, dtype=np.int32)
        A = np.zeros((len(mons), kmax), dtype=np.int32)
        K = np.zeros(len(mons), dtype=np.int64)
        for r, (p, a) in enumerate(mons):
            S[r, :len(p)] = p
            A[r, :len(a)] = a
            K[r] = len(p)
        rows.append((S, A, K))
    return _assemble(n, rows, np.asarray(coef, dtype=np.float64).reshape(-1, 4), dict(explicit=True))


def gaussian_int_cdd(rng, size, lo=-3, hi=3, nonzero=True):
    """Complex numbers with integer parts in [lo, hi] as double-doubles with
    zero low words; ``nonzero`` redraws exact zeros."""
    out = np.zeros((size, 4))
    re = rng.integers(lo, hi + 1, size=size)
    im = rng.integers(lo, hi + 1, size=size)
    if nonzero:
        while True:
            z = (re == 0) & (im == 0)
            if not z.any():
                break
            re[z] = rng.integers(lo, hi + 1, size=z.sum())
            im[z] = rng.integers(lo, hi + 1, size=z.sum())
    out[:, 0] = re
    out[:, 2] = im
    return out


def dense_system(seed, n, degrees):
    """A square system whose polynomial i holds every monomial of total
    degree <= degrees[i] in the n variables (the constant included), with
    random complex double-double coefficients near the unit circle: generic,
    so the total-degree homotopy has prod(degrees) finite regular solutions
    (with probability one)."""
    import itertools

    rng = np.random.Generator(np.random.PCG64(seed))
    polys = []
    for d in degrees:
        mons = []
        for e in itertools.product(range(d + 1), repeat=n):
            if sum(e) <= d:
                pos = [v for v in range(n) if e[v] > 0]
                mons.append((pos, [e[v] for v in pos]))
        polys.append(mons)
    M = sum(len(p) for p in polys)
    return from_monomials(n, polys, random_cdd(rng, M))

