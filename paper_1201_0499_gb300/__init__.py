"""GB300-native evaluation of sparse polynomial systems and their Jacobians
(Verschelde & Yoffe, "Evaluating polynomials in several variables and their
derivatives on a GPU computing processor").

The computation lives in the CUDA library ``libpolyeval.so`` (sources in
``csrc/``, C ABI in ``include/polyeval.h``); this package is its thin Python
binding.  Build the library with ``paper_1201_0499_gb300.build.build()``.
"""
from ._binding import (  # noqa: F401
    LIB_PATH,
    PE_ALLOW_ZERO_COEF,
    PE_DD,
    PE_DD_INT,
    PE_ECUDA,
    PE_EDEVICE,
    PE_EINVAL,
    PE_ENOMEM,
    PE_ERANGE,
    PE_F64,
    PE_MAX_EXP,
    PE_MAX_VARS,
    PE_OK,
    PE_PAPER_KERNELS,
    PE_QD_INT,
    PolyEval,
    PolyEvalError,
    PolyEvalMany,
    load_library,
    pe_system,
    polyeval_autotune,
    polyeval_cost,
    polyeval_create,
    polyeval_create_many,
    polyeval_destroy,
    polyeval_eval,
    polyeval_eval_host,
    polyeval_eval_many,
    polyeval_eval_noalloc,
    polyeval_fp64_peak,
    polyeval_newton,
    polyeval_many_layout,
    polyeval_status,
    polyeval_strerror,
    polyeval_timing,
    polyeval_timing_read,
    polyeval_validate,
)
