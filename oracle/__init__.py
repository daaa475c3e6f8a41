"""Oracles for the polynomial-system evaluation -- TEST INFRASTRUCTURE ONLY.

* ``oracle.exact``: exact (dyadic-rational) evaluation of the definitions of
  Section 2, Eq. (1); the ground truth every parity test measures against.
* ``oracle.dd``: a plain C double-double evaluator of the same definitions
  (``dd_oracle.c``), used for whole-batch comparisons and as the timed CPU
  baseline.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The product path never does.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dd_oracle.c")
_LIB = os.path.join(_HERE, "_dd_oracle.so")
_lib = None


def build_command():
    return ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", _LIB, _SRC, "-lm"]


def build(force: bool = False) -> str:
    """Compile the C oracle in place (the checker is built, not used)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.run(build_command(), check=True)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        lib.dd_oracle_eval.argtypes = [ctypes.c_int32, ctypes.c_int32, P, P, P, P, P, P, ctypes.c_int64,
                                       ctypes.c_int64, ctypes.c_int64, P, P, ctypes.c_int32]
        lib.dd_oracle_eval.restype = ctypes.c_int
        lib.dd_oracle_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def max_threads() -> int:
    return int(_load().dd_oracle_max_threads())


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def dd_eval(system, pts, q0: int = 0, q1=None, threads: int = 0, out=None):
    """C double-double oracle on points [q0, q1).  Returns (f [N,P,4], J [N,n,P,4])
    with the requested points filled (the rest zero, or whatever ``out`` held)."""
    lib = _load()
    n, N = system.n_vars, system.n_polys
    P = pts.shape[1]
    q1 = P if q1 is None else q1
    pts = np.ascontiguousarray(pts, dtype=np.float64)
    if out is None:
        f = np.zeros((N, P, 4))
        J = np.zeros((N, n, P, 4))
    else:
        f, J = out
    arrs = [np.ascontiguousarray(system.poly_ptr, dtype=np.int64), np.ascontiguousarray(system.mono_ptr, dtype=np.int64),
            np.ascontiguousarray(system.pos, dtype=np.int32), np.ascontiguousarray(system.exp, dtype=np.int32),
            np.ascontiguousarray(system.coef, dtype=np.float64)]
    rc = lib.dd_oracle_eval(n, N, *[_ptr(a) for a in arrs], _ptr(pts), P, q0, q1, _ptr(f), _ptr(J), threads)
    if rc != 0:
        raise ValueError(f"dd_oracle_eval failed ({rc})")
    return f, J
