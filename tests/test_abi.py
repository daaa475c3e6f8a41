"""The C ABI without a GPU: the library loads, exports every entry point the
header declares, and host-side validation rejects malformed systems
(Section 2, Eq. 1: sparse monomials with sorted positions, exponents >= 1,
nonzero coefficients)."""
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def pkg():
    import paper_1201_0499_gb300 as pkg
    from paper_1201_0499_gb300 import build

    build.build()
    pkg.load_library()
    return pkg


def declared_entry_points():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            names += re.findall(r"^PE_API\s+[\w\s\*]*?\b(polyeval_\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_entry_points()
    for required in ["polyeval_create", "polyeval_eval", "polyeval_destroy", "polyeval_create_many",
                     "polyeval_eval_many", "polyeval_status", "polyeval_strerror", "polyeval_validate"]:
        assert required in names


def test_library_exports_every_declared_symbol(pkg):
    lib = pkg.load_library()
    for name in declared_entry_points():
        assert hasattr(lib, name), name
    # and the binding has a function of the same name for each
    for name in declared_entry_points():
        assert hasattr(pkg, name), name


def test_strerror(pkg):
    assert pkg.polyeval_strerror(pkg.PE_OK) == "ok"
    for c in (pkg.PE_EINVAL, pkg.PE_ENOMEM, pkg.PE_ECUDA, pkg.PE_ERANGE, pkg.PE_EDEVICE):
        assert pkg.polyeval_strerror(c) != "unknown status code"
    assert pkg.polyeval_strerror(12345) == "unknown status code"


def _small():
    return synth.from_monomials(4, [[([0, 2], [3, 1]), ([1], [2])], [([], []), ([0, 1, 2, 3], [1, 1, 1, 1])]],
                                [[1, 0, 0.5, 0], [2, 0, 0, 0], [0, 0, 1, 0], [1, 1e-17, -1, 0]])


def _mutate(s, **kw):
    import copy

    t = copy.deepcopy(s)
    for k, v in kw.items():
        setattr(t, k, v)
    return t


def test_validate_accepts_good_systems(pkg):
    assert pkg.polyeval_validate(_small()) == pkg.PE_OK
    s, _ = synth.config(1)
    assert pkg.polyeval_validate(s) == pkg.PE_OK
    empty = synth.from_monomials(3, [], np.zeros((0, 4)))
    assert pkg.polyeval_validate(empty) == pkg.PE_OK


def test_validate_rejects(pkg):
    s = _small()
    E, R = pkg.PE_EINVAL, pkg.PE_ERANGE
    assert pkg.polyeval_validate(_mutate(s, n_vars=0)) == E
    assert pkg.polyeval_validate(_mutate(s, n_vars=70000)) == R
    pos = s.pos.copy(); pos[0] = 4
    assert pkg.polyeval_validate(_mutate(s, pos=pos)) == E          # position >= n
    pos = s.pos.copy(); pos[0], pos[1] = pos[1], pos[0]
    assert pkg.polyeval_validate(_mutate(s, pos=pos)) == E          # not increasing
    pos = s.pos.copy(); pos[1] = pos[0]
    assert pkg.polyeval_validate(_mutate(s, pos=pos)) == E          # duplicate position
    pos = s.pos.copy(); pos[0] = -1
    assert pkg.polyeval_validate(_mutate(s, pos=pos)) == E
    ex = s.exp.copy(); ex[0] = 0
    assert pkg.polyeval_validate(_mutate(s, exp=ex)) == E           # exponent 0
    ex = s.exp.copy(); ex[0] = 257
    assert pkg.polyeval_validate(_mutate(s, exp=ex)) == R           # above PE_MAX_EXP
    ex = s.exp.copy(); ex[0] = 256
    assert pkg.polyeval_validate(_mutate(s, exp=ex)) == pkg.PE_OK
    c = s.coef.copy(); c[1] = 0
    assert pkg.polyeval_validate(_mutate(s, coef=c)) == E           # c = 0 (Eq. 1 asks c != 0)
    assert pkg.polyeval_validate(_mutate(s, coef=c), pkg.PE_ALLOW_ZERO_COEF) == pkg.PE_OK
    c = s.coef.copy(); c[0, 1] = np.nan
    assert pkg.polyeval_validate(_mutate(s, coef=c)) == E
    pp = s.poly_ptr.copy(); pp[0] = 1
    assert pkg.polyeval_validate(_mutate(s, poly_ptr=pp)) == E
    mp = s.mono_ptr.copy(); mp[2] = mp[1] - 1
    assert pkg.polyeval_validate(_mutate(s, mono_ptr=mp)) == E


C_PROGRAM = r"""
#include <stdint.h>
#include <stdio.h>
#include "polyeval.h"

int main(void) {
  /* f_0 = x0^2 x1 + 3, f_1 = (1 + 2i) x1 (two variables, two polynomials) */
  const int64_t poly_ptr[3] = {0, 2, 3};
  const int64_t mono_ptr[4] = {0, 2, 2, 3};
  const int32_t pos[3] = {0, 1, 1};
  int32_t expo[3] = {2, 1, 1};
  const pe_cdd coef[3] = {{1.0, 0.0, 0.0, 0.0}, {3.0, 0.0, 0.0, 0.0}, {1.0, 0.0, 2.0, 0.0}};
  pe_system s;
  s.n_vars = 2;
  s.n_polys = 2;
  s.poly_ptr = poly_ptr;
  s.mono_ptr = mono_ptr;
  s.pos = pos;
  s.exp = expo;
  s.coef = coef;
  s.coef_qd = NULL;
  const int good = polyeval_validate(&s, 0);
  expo[2] = 0; /* exponent < 1 */
  const int bad = polyeval_validate(&s, 0);
  polyeval_destroy(NULL); /* NULL-safe */
  printf("%d %d %s\n", good, bad, polyeval_strerror(bad));
  return (good == PE_OK && bad == PE_EINVAL) ? 0 : 1;
}
"""


def test_header_is_c99_and_library_links_from_c(pkg, tmp_path):
    """A plain C99 program includes the header (warnings are errors), links
    against the library and calls the host-only entry points."""
    import shutil
    import subprocess

    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lib_dir = os.path.join(ROOT, "paper_1201_0499_gb300")
    src = tmp_path / "abi.c"
    exe = tmp_path / "abi"
    src.write_text(C_PROGRAM)
    subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", lib_dir, "-lpolyeval", f"-Wl,-rpath,{lib_dir}"],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stdout + out.stderr
    assert out.stdout.split()[:2] == ["0", str(pkg.PE_EINVAL)]


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    """Without the built library every entry point raises: there is no CPU
    fallback behind the binding."""
    import paper_1201_0499_gb300 as pkg
    from paper_1201_0499_gb300 import _binding

    monkeypatch.setattr(_binding, "_lib", None)
    monkeypatch.setattr(_binding, "LIB_PATH", str(tmp_path / "libpolyeval.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pkg.load_library()
    with pytest.raises(RuntimeError, match="not built"):
        pkg.polyeval_validate(_small())
    with pytest.raises(RuntimeError, match="not built"):
        pkg.PolyEval(_small(), pkg.PE_DD, max_points=4)


def test_track_defaults_host_only(pkg):
    """polyeval_track_defaults runs on the host: the documented defaults per
    precision, and PE_EINVAL for a precision the tracker does not take."""
    import cmath

    lo, hi = pkg.polyeval_track_defaults(pkg.PE_F64), pkg.polyeval_track_defaults(pkg.PE_DD)
    for prm in (lo, hi):
        assert complex(prm.gamma_re, prm.gamma_im) == pytest.approx(cmath.exp(1j), abs=1e-15)
        assert 0 < prm.h_min < prm.h_init <= prm.h_max <= 1.0
        assert prm.corr_tol == 1e-6 and prm.max_corr == 3 and prm.succ_grow == 3
        assert prm.max_iters >= 1 and prm.x_big > 1.0
    assert hi.end_tol < lo.end_tol and hi.h_min < lo.h_min
    assert (lo.mixed, hi.mixed) == (0, 1)
    assert pkg.polyeval_track_defaults(pkg.PE_DD_INT).end_tol == hi.end_tol
    for bad in (pkg.PE_QD_INT, 99):
        with pytest.raises(pkg.PolyEvalError) as e:
            pkg.polyeval_track_defaults(bad)
        assert e.value.code == pkg.PE_EINVAL


def test_noalloc_argument_checks_before_any_cuda_call(pkg):
    """polyeval_eval_noalloc checks its arguments on the host before it
    touches the device: these calls return without a GPU.  The addresses are
    never dereferenced on these paths (16 is merely aligned, 24 is not)."""
    def sysd(n=4, N=2, addr=16):
        return pkg.pe_system(n, N, addr, addr, addr, addr, addr, None)

    def call(s, max_k=4, max_exp=3, points=16, P=8, f=16, J=16):
        try:
            pkg.polyeval_eval_noalloc(s, max_k, max_exp, points, P, f, J)
            return pkg.PE_OK
        except pkg.PolyEvalError as e:
            return e.code

    assert call(sysd(), P=0) == pkg.PE_OK                      # nothing to evaluate
    assert call(sysd(N=0)) == pkg.PE_OK
    assert call(sysd(n=0)) == pkg.PE_EINVAL                    # no variables
    assert call(sysd(), P=-1) == pkg.PE_EINVAL
    assert call(sysd(), max_exp=0) == pkg.PE_EINVAL
    assert call(sysd(), max_exp=pkg.PE_MAX_EXP + 1) == pkg.PE_ERANGE
    assert call(sysd(n=pkg.PE_MAX_VARS + 1)) == pkg.PE_ERANGE
    assert call(sysd(), points=None) == pkg.PE_EINVAL           # null arrays
    assert call(sysd(addr=0)) == pkg.PE_EINVAL
    assert call(sysd(), points=24) == pkg.PE_EINVAL             # misaligned
    assert call(sysd(), f=24) == pkg.PE_EINVAL
    assert call(sysd(n=64), max_exp=200, P=100000) == pkg.PE_ERANGE  # power table above the static scratch


def test_null_handle_and_bad_create_arguments_without_a_gpu(pkg):
    """Every entry point that takes a handle answers PE_EINVAL for a NULL one,
    and polyeval_create rejects bad arguments before any CUDA call."""
    import ctypes

    lib = pkg.load_library()
    N = None
    calls = {
        "polyeval_eval": (N, N, 4, N, N, N),
        "polyeval_eval_host": (N, N, 4, N, N, N),
        "polyeval_autotune": (N, N, 4, N, N, N, N, N, N),
        "polyeval_set_launch": (N, 4, 1, 1, 1),
        "polyeval_newton": (N, N, 4, N, N, N, N),
        "polyeval_eval_many": (N, N, N, N, N),
        "polyeval_many_layout": (N, 0, N, N, N),
        "polyeval_cost": (N, N, N),
        "polyeval_timing": (N, 1),
        "polyeval_timing_read": (N, N, N, N),
        "polyeval_status": (N,),
        "polyeval_bezout": (N, N, N),
        "polyeval_start_points": (N, 0, 4, N, N),
        "polyeval_track": (N, N, N, 4, N, N, N, N),
        "polyeval_track_adaptive": (N, N, N, N, N, 4, N, N, N),
    }
    assert set(calls) | {"polyeval_destroy"} >= {n for n in declared_entry_points()
                                                  if n not in ("polyeval_validate", "polyeval_create",
                                                               "polyeval_create_many", "polyeval_strerror",
                                                               "polyeval_fp64_peak", "polyeval_eval_noalloc",
                                                               "polyeval_track_defaults")}
    for name, args in calls.items():
        assert getattr(lib, name)(*args) == pkg.PE_EINVAL, name
    lib.polyeval_destroy(None)

    s = pkg.pe_system()  # all zero: n_vars = 0 is invalid
    out = ctypes.c_void_p()
    assert lib.polyeval_create(None, pkg.PE_DD, 0, 4, ctypes.byref(out)) == pkg.PE_EINVAL
    assert lib.polyeval_create(ctypes.byref(s), pkg.PE_DD, 0, 4, None) == pkg.PE_EINVAL
    assert lib.polyeval_create(ctypes.byref(s), 77, 0, 4, ctypes.byref(out)) == pkg.PE_EINVAL
    assert lib.polyeval_create(ctypes.byref(s), pkg.PE_DD, 0, 0, ctypes.byref(out)) == pkg.PE_EINVAL
    assert lib.polyeval_create(ctypes.byref(s), pkg.PE_DD, 0, 4, ctypes.byref(out)) == pkg.PE_EINVAL  # n_vars 0
    assert out.value is None
