"""ctypes binding of the C ABI in ``include/polyeval.h``.

Argument marshalling only: every step of the evaluation runs in the CUDA
library ``libpolyeval.so``.  If the library is missing or fails to load,
every call raises -- there is no CPU fallback.

Functions keep the C names (``polyeval_create``, ``polyeval_eval``, ...).
Device buffers may be given as torch CUDA tensors or as raw integer
addresses; streams as ``torch.cuda.Stream``, raw ``cudaStream_t`` integers or
None (the current torch stream when torch is loaded, else the legacy default
stream).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

PE_OK = 0
PE_EINVAL = -1
PE_ENOMEM = -2
PE_ECUDA = -3
PE_ERANGE = -4
PE_EDEVICE = -5

PE_DD = 0
PE_F64 = 1
PE_DD_INT = 2
PE_QD_INT = 3

PE_ALLOW_ZERO_COEF = 1
PE_PAPER_KERNELS = 2

PE_MAX_VARS = 65535
PE_MAX_EXP = 256

PE_PATH_RUNNING = 0
PE_PATH_SUCCESS = 1
PE_PATH_FAILED = 2
PE_PATH_DIVERGED = 3
PE_PATH_END_NOT_CONVERGED = 4

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libpolyeval.so")

_lib = None


class PolyEvalError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__(f"{where}: {code} ({polyeval_strerror(code)})" if where else f"{code}")


class pe_system(ctypes.Structure):
    _fields_ = [
        ("n_vars", ctypes.c_int32),
        ("n_polys", ctypes.c_int32),
        ("poly_ptr", ctypes.c_void_p),
        ("mono_ptr", ctypes.c_void_p),
        ("pos", ctypes.c_void_p),
        ("exp", ctypes.c_void_p),
        ("coef", ctypes.c_void_p),
        ("coef_qd", ctypes.c_void_p),
    ]


class pe_track_params(ctypes.Structure):
    _fields_ = [
        ("gamma_re", ctypes.c_double),
        ("gamma_im", ctypes.c_double),
        ("h_init", ctypes.c_double),
        ("h_min", ctypes.c_double),
        ("h_max", ctypes.c_double),
        ("corr_tol", ctypes.c_double),
        ("end_tol", ctypes.c_double),
        ("x_big", ctypes.c_double),
        ("max_corr", ctypes.c_int32),
        ("max_end", ctypes.c_int32),
        ("succ_grow", ctypes.c_int32),
        ("mixed", ctypes.c_int32),
        ("max_iters", ctypes.c_int64),
    ]


def load_library(path: Optional[str] = None):
    """Load libpolyeval.so (once).  Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built: run `python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    D = ctypes.POINTER(ctypes.c_double)
    sig = {
        "polyeval_validate": ([ctypes.POINTER(pe_system), U32], ctypes.c_int),
        "polyeval_create": ([ctypes.POINTER(pe_system), ctypes.c_int, U32, I64, ctypes.POINTER(P)], ctypes.c_int),
        "polyeval_eval": ([P, P, I64, P, P, P], ctypes.c_int),
        "polyeval_eval_host": ([P, P, I64, P, P, P], ctypes.c_int),
        "polyeval_create_many": ([ctypes.POINTER(pe_system), I32, ctypes.c_int, U32, ctypes.POINTER(I64),
                                  ctypes.POINTER(P)], ctypes.c_int),
        "polyeval_many_layout": ([P, I32, ctypes.POINTER(I64), ctypes.POINTER(I64), ctypes.POINTER(I64)],
                                 ctypes.c_int),
        "polyeval_eval_many": ([P, P, P, P, P], ctypes.c_int),
        "polyeval_cost": ([P, D, D], ctypes.c_int),
        "polyeval_timing": ([P, ctypes.c_int], ctypes.c_int),
        "polyeval_timing_read": ([P, D, ctypes.POINTER(I64), ctypes.POINTER(I64)], ctypes.c_int),
        "polyeval_status": ([P], ctypes.c_int),
        "polyeval_destroy": ([P], None),
        "polyeval_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "polyeval_fp64_peak": ([P, D, D], ctypes.c_int),
        "polyeval_eval_noalloc": ([ctypes.POINTER(pe_system), I32, I32, P, I64, P, P, P], ctypes.c_int),
        "polyeval_newton": ([P, P, I64, P, P, P, P], ctypes.c_int),
        "polyeval_autotune": ([P, P, I64, P, P, P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                               ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
        "polyeval_set_launch": ([P, I64, ctypes.c_int, ctypes.c_int, ctypes.c_int], ctypes.c_int),
        "polyeval_track_defaults": ([ctypes.c_int, ctypes.POINTER(pe_track_params)], ctypes.c_int),
        "polyeval_bezout": ([P, D, ctypes.POINTER(I32)], ctypes.c_int),
        "polyeval_start_points": ([P, I64, I64, P, P], ctypes.c_int),
        "polyeval_track": ([P, ctypes.POINTER(pe_track_params), P, I64, P, P, ctypes.POINTER(I64), P], ctypes.c_int),
        "polyeval_track_adaptive": ([P, P, ctypes.POINTER(pe_track_params), ctypes.POINTER(pe_track_params), P, I64,
                                     P, ctypes.POINTER(I64), P], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = res
    _lib = lib
    return lib


def _addr(x) -> Optional[int]:
    """Device/host address of a tensor, ndarray or integer."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> Optional[int]:
    if s is None:
        try:
            import torch

            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(rc: int, where: str):
    if rc != PE_OK:
        raise PolyEvalError(rc, where)


class _Packed:
    """A pe_system plus the numpy arrays it points into.  ``system.coef`` is
    [M, 4] (complex double-double) or [M, 8] (complex quad-double: passed as
    coef_qd, with its leading two parts per component as coef)."""

    def __init__(self, system):
        coef = np.asarray(system.coef, dtype=np.float64)
        coef = coef.reshape(-1, coef.shape[-1] if coef.ndim == 2 and coef.shape[-1] in (4, 8) else 4)
        qd = None
        if coef.shape[1] == 8:
            qd = np.ascontiguousarray(coef)
            coef = coef[:, [0, 1, 4, 5]]
        self.arrays = [
            np.ascontiguousarray(system.poly_ptr, dtype=np.int64),
            np.ascontiguousarray(system.mono_ptr, dtype=np.int64),
            np.ascontiguousarray(system.pos, dtype=np.int32),
            np.ascontiguousarray(system.exp, dtype=np.int32),
            np.ascontiguousarray(coef),
        ]
        self.qd = qd
        a = self.arrays
        self.struct = pe_system(int(system.n_vars), int(system.n_polys), *[x.ctypes.data for x in a],
                                qd.ctypes.data if qd is not None else None)


# ----------------------------------------------------------------------------
# the C ABI, one Python function per entry point
# ----------------------------------------------------------------------------

def polyeval_strerror(code: int) -> str:
    return load_library().polyeval_strerror(int(code)).decode()


def polyeval_validate(system, flags: int = 0) -> int:
    """Host-only check of a system; returns the status code (does not raise)."""
    pk = _Packed(system)
    return int(load_library().polyeval_validate(ctypes.byref(pk.struct), flags))


def polyeval_create(system, precision: int = PE_DD, flags: int = 0, max_points: int = 1) -> int:
    pk = _Packed(system)
    h = ctypes.c_void_p()
    _check(load_library().polyeval_create(ctypes.byref(pk.struct), precision, flags, max_points, ctypes.byref(h)),
           "polyeval_create")
    return int(h.value)


def polyeval_create_many(systems: Sequence, points_per_system: Sequence[int], precision: int = PE_DD,
                         flags: int = 0) -> int:
    packs = [_Packed(s) for s in systems]
    arr = (pe_system * len(packs))(*[p.struct for p in packs])
    pps = (ctypes.c_int64 * len(packs))(*[int(v) for v in points_per_system])
    h = ctypes.c_void_p()
    _check(load_library().polyeval_create_many(arr, len(packs), precision, flags, pps, ctypes.byref(h)),
           "polyeval_create_many")
    return int(h.value)


def polyeval_eval(h: int, points, P: int, out_f, out_J, stream=None) -> None:
    _check(load_library().polyeval_eval(h, _addr(points), int(P), _addr(out_f), _addr(out_J), _stream(stream)),
           "polyeval_eval")


def polyeval_autotune(h: int, points, P: int, out_f, out_J, stream=None):
    """Time the launch candidates for P points and keep the fastest in the
    handle; returns (chunks, shape, groups)."""
    c, m, g = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(load_library().polyeval_autotune(h, _addr(points), int(P), _addr(out_f), _addr(out_J), _stream(stream),
                                            ctypes.byref(c), ctypes.byref(m), ctypes.byref(g)), "polyeval_autotune")
    return c.value, m.value, g.value


def polyeval_set_launch(h: int, P: int, chunks: int = 0, shape: int = 0, groups: int = 0) -> None:
    """Fix the launch for calls with P points (0 = built-in choice)."""
    _check(load_library().polyeval_set_launch(h, int(P), int(chunks), int(shape), int(groups)), "polyeval_set_launch")


def polyeval_newton(h: int, points, P: int, out_f, out_J, norms=None, stream=None) -> None:
    """One Newton step at P points (points updated in place; out_f receives dx)."""
    _check(load_library().polyeval_newton(h, _addr(points), int(P), _addr(out_f), _addr(out_J), _addr(norms),
                                          _stream(stream)), "polyeval_newton")


def polyeval_eval_host(h: int, points, P: int, out_f, out_J, stream=None) -> None:
    _check(load_library().polyeval_eval_host(h, _addr(points), int(P), _addr(out_f), _addr(out_J), _stream(stream)),
           "polyeval_eval_host")


def polyeval_many_layout(h: int, s: int):
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().polyeval_many_layout(h, s, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
           "polyeval_many_layout")
    return a.value, b.value, c.value


def polyeval_eval_many(h: int, points, out_f, out_J, stream=None) -> None:
    _check(load_library().polyeval_eval_many(h, _addr(points), _addr(out_f), _addr(out_J), _stream(stream)),
           "polyeval_eval_many")


def polyeval_cost(h: int):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().polyeval_cost(h, ctypes.byref(a), ctypes.byref(b)), "polyeval_cost")
    return a.value, b.value


def polyeval_timing(h: int, enable: bool) -> None:
    _check(load_library().polyeval_timing(h, int(bool(enable))), "polyeval_timing")


def polyeval_timing_read(h: int):
    """(summed main-kernel ms, timed launches, kernels queued) since polyeval_timing."""
    ms, n, k = ctypes.c_double(), ctypes.c_int64(), ctypes.c_int64()
    _check(load_library().polyeval_timing_read(h, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(k)),
           "polyeval_timing_read")
    return ms.value, n.value, k.value


def polyeval_status(h: int) -> int:
    return int(load_library().polyeval_status(h))


def polyeval_destroy(h: Optional[int]) -> None:
    load_library().polyeval_destroy(h)


def polyeval_fp64_peak(stream=None):
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load_library().polyeval_fp64_peak(_stream(stream), ctypes.byref(a), ctypes.byref(b)), "polyeval_fp64_peak")
    return a.value, b.value


def polyeval_eval_noalloc(dev_sys: pe_system, max_k: int, max_exp: int, points, P: int, out_f, out_J,
                          stream=None) -> None:
    """For callers that cannot let the library allocate device memory:
    ``dev_sys`` is a pe_system whose array fields hold device addresses (for
    example of torch tensors the caller owns); scratch comes from a static
    device array inside the library."""
    _check(load_library().polyeval_eval_noalloc(ctypes.byref(dev_sys), int(max_k), int(max_exp), _addr(points),
                                                int(P), _addr(out_f), _addr(out_J), _stream(stream)),
           "polyeval_eval_noalloc")


def polyeval_track_defaults(precision: int) -> pe_track_params:
    prm = pe_track_params()
    _check(load_library().polyeval_track_defaults(precision, ctypes.byref(prm)), "polyeval_track_defaults")
    return prm


def polyeval_bezout(h: int, n: int):
    """(number of paths, [d_0, ..., d_{n-1}])."""
    c = ctypes.c_double()
    d = (ctypes.c_int32 * n)()
    _check(load_library().polyeval_bezout(h, ctypes.byref(c), d), "polyeval_bezout")
    return c.value, list(d)


def polyeval_start_points(h: int, first: int, P: int, points, stream=None) -> None:
    _check(load_library().polyeval_start_points(h, int(first), int(P), _addr(points), _stream(stream)),
           "polyeval_start_points")


def polyeval_track(h: int, prm: pe_track_params, points, P: int, t=None, status=None, stream=None) -> int:
    """Track P paths in place; returns the number of iterations."""
    it = ctypes.c_int64()
    _check(load_library().polyeval_track(h, ctypes.byref(prm), _addr(points), int(P), _addr(t), _addr(status),
                                         ctypes.byref(it), _stream(stream)), "polyeval_track")
    return it.value


def polyeval_track_adaptive(h_lo: int, h_hi: int, prm_lo: pe_track_params, prm_hi: pe_track_params, points, P: int,
                            status, stream=None) -> int:
    """Track in double, refine or re-track in double-double; returns the
    number of paths tracked again in double-double."""
    esc = ctypes.c_int64()
    _check(load_library().polyeval_track_adaptive(h_lo, h_hi, ctypes.byref(prm_lo), ctypes.byref(prm_hi),
                                                  _addr(points), int(P), _addr(status), ctypes.byref(esc),
                                                  _stream(stream)), "polyeval_track_adaptive")
    return esc.value


# ----------------------------------------------------------------------------
# convenience wrappers over torch device memory
# ----------------------------------------------------------------------------

def _elem(precision: int) -> int:
    """Doubles per complex element of a precision."""
    return 2 if precision == PE_F64 else 8 if precision == PE_QD_INT else 4


class PolyEval:
    """One compiled system.  ``eval(points)`` takes a float64 CUDA tensor of
    shape [n, P, c] -- c = 4 (double-double), 8 (quad-double) or 2 (double)
    -- and returns (f [N, P, c], J [N, n, P, c]) as new CUDA tensors."""

    def __init__(self, system, precision: int = PE_DD, max_points: int = 1, flags: int = 0):
        self.n_vars = int(system.n_vars)
        self.n_polys = int(system.n_polys)
        self.precision = precision
        self.max_points = int(max_points)
        self.handle = polyeval_create(system, precision, flags, max_points)

    def eval(self, points, out_f=None, out_J=None, stream=None):
        import torch

        c = _elem(self.precision)
        if points.dtype != torch.float64 or not points.is_cuda or tuple(points.shape[::2]) != (self.n_vars, c):
            raise ValueError(f"points must be a float64 CUDA tensor of shape [{self.n_vars}, P, {c}]")
        points = points.contiguous()
        P = points.shape[1]
        if out_f is None:
            out_f = torch.empty((self.n_polys, P, c), dtype=torch.float64, device=points.device)
        if out_J is None:
            out_J = torch.empty((self.n_polys, self.n_vars, P, c), dtype=torch.float64, device=points.device)
        polyeval_eval(self.handle, points, P, out_f, out_J, stream)
        return out_f, out_J

    def autotune(self, points, out_f=None, out_J=None, stream=None):
        """Tune the launch for this point count; returns (chunks, shape, groups)."""
        import torch

        c = _elem(self.precision)
        P = points.shape[1]
        if out_f is None:
            out_f = torch.empty((self.n_polys, P, c), dtype=torch.float64, device=points.device)
        if out_J is None:
            out_J = torch.empty((self.n_polys, self.n_vars, P, c), dtype=torch.float64, device=points.device)
        return polyeval_autotune(self.handle, points.contiguous(), P, out_f, out_J, stream)

    def newton(self, points, out_dx=None, out_J=None, norms=None, stream=None):
        """One Newton step; ``points`` (CUDA tensor [n, P, c]) is updated in
        place.  Returns (dx, LU, norms [P, 2])."""
        import torch

        c = _elem(self.precision)
        P = points.shape[1]
        if out_dx is None:
            out_dx = torch.empty((self.n_polys, P, c), dtype=torch.float64, device=points.device)
        if out_J is None:
            out_J = torch.empty((self.n_polys, self.n_vars, P, c), dtype=torch.float64, device=points.device)
        if norms is None:
            norms = torch.empty((P, 2), dtype=torch.float64, device=points.device)
        polyeval_newton(self.handle, points, P, out_dx, out_J, norms, stream)
        return out_dx, out_J, norms

    def cost(self):
        return polyeval_cost(self.handle)

    def bezout(self):
        """(number of paths of the total-degree homotopy, degrees)."""
        return polyeval_bezout(self.handle, self.n_vars)

    def start_points(self, P: int, first: int = 0, device="cuda", stream=None):
        """Start solutions of paths first .. first + P - 1 as a CUDA tensor [n, P, c]."""
        import torch

        x = torch.empty((self.n_vars, P, _elem(self.precision)), dtype=torch.float64, device=device)
        polyeval_start_points(self.handle, first, P, x, stream)
        return x

    def track(self, points, prm: Optional[pe_track_params] = None, stream=None):
        """Track the paths starting at ``points`` (updated in place to the end
        points); returns (status [P] int32, t [P], iterations)."""
        import torch

        P = points.shape[1]
        prm = prm or polyeval_track_defaults(self.precision)
        status = torch.empty(P, dtype=torch.int32, device=points.device)
        t = torch.empty(P, dtype=torch.float64, device=points.device)
        it = polyeval_track(self.handle, prm, points, P, t, status, stream)
        return status, t, it

    def status(self) -> int:
        return polyeval_status(self.handle)

    def close(self):
        if self.handle:
            polyeval_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class PolyEvalMany:
    """A batch of systems evaluated in one launch, each at its own points.
    ``eval(points_list)`` takes a list of float64 CUDA tensors [n_s, P_s, c]
    and returns lists of (f_s, J_s) views into the batch output buffers."""

    def __init__(self, systems, points_per_system, precision: int = PE_DD, flags: int = 0):
        self.shapes = [(int(s.n_vars), int(s.n_polys), int(P)) for s, P in zip(systems, points_per_system)]
        self.precision = precision
        self.handle = polyeval_create_many(systems, points_per_system, precision, flags)
        self.layout = [polyeval_many_layout(self.handle, s) for s in range(len(systems) + 1)]

    def buffers(self, device="cuda"):
        import torch

        c = _elem(self.precision)
        tot = self.layout[-1]
        return (torch.empty((tot[0], c), dtype=torch.float64, device=device),
                torch.empty((tot[1], c), dtype=torch.float64, device=device),
                torch.empty((tot[2], c), dtype=torch.float64, device=device))

    def pack_points(self, points_list, buf):
        c = _elem(self.precision)
        for (n, N, P), (po, _fo, _jo), x in zip(self.shapes, self.layout, points_list):
            buf[po:po + n * P].view(n, P, c).copy_(x)

    def views(self, out_f, out_J):
        c = _elem(self.precision)
        fs, Js = [], []
        for (n, N, P), (_po, fo, jo) in zip(self.shapes, self.layout):
            fs.append(out_f[fo:fo + N * P].view(N, P, c))
            Js.append(out_J[jo:jo + N * n * P].view(N, n, P, c))
        return fs, Js

    def eval_buffers(self, pts_buf, f_buf, J_buf, stream=None):
        polyeval_eval_many(self.handle, pts_buf, f_buf, J_buf, stream)

    def eval(self, points_list, stream=None):
        pts_buf, f_buf, J_buf = self.buffers(points_list[0].device)
        self.pack_points(points_list, pts_buf)
        self.eval_buffers(pts_buf, f_buf, J_buf, stream)
        return self.views(f_buf, J_buf)

    def autotune(self, pts_buf, f_buf, J_buf, stream=None):
        """Tune the batch launch on the packed buffers; returns (chunks, shape, groups)."""
        return polyeval_autotune(self.handle, pts_buf, 0, f_buf, J_buf, stream)

    def set_launch(self, chunks: int = 0, shape: int = 0, groups: int = 0):
        polyeval_set_launch(self.handle, 0, chunks, shape, groups)

    def cost(self):
        return polyeval_cost(self.handle)

    def close(self):
        if self.handle:
            polyeval_destroy(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
