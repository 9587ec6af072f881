"""ctypes declarations of the liblrfg C ABI (include/lrfg.h).  Argument marshalling only."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblrfg.so")

LRFG_OK, LRFG_EINVAL, LRFG_ENOMEM, LRFG_ENOCONV, LRFG_ECUDA, LRFG_ETIMEOUT, LRFG_ENOTSUP = range(7)
LRFG_FULL, LRFG_CP, LRFG_TUCKER, LRFG_TT = 0, 1, 2, 3
LRFG_FP64, LRFG_MIXED = 0, 1
LRFG_GANI, LRFG_GA = 0, 1
LRFG_MUL_IDENTITY, LRFG_MUL_DERIV, LRFG_MUL_GAUSS = 0, 1, 2

STATUS_NAMES = {0: "LRFG_OK", 1: "LRFG_EINVAL", 2: "LRFG_ENOMEM", 3: "LRFG_ENOCONV", 4: "LRFG_ECUDA",
                5: "LRFG_ETIMEOUT", 6: "LRFG_ENOTSUP"}


class lrfg_tt(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int * 3), ("r", C.c_int * 4), ("cores", C.c_void_p * 3)]


class lrfg_tucker(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int * 3), ("r", C.c_int * 3), ("core", C.c_void_p),
                ("factors", C.c_void_p * 3)]


class lrfg_coeff(C.Structure):
    _fields_ = [("d", C.c_int), ("N", C.c_int * 3), ("fmt", C.c_int), ("values", C.c_void_p),
                ("tt", lrfg_tt), ("on_device", C.c_int), ("tk", lrfg_tucker), ("B", C.c_double * 9)]


class lrfg_opts(C.Structure):
    _fields_ = [("fmt", C.c_int), ("prec", C.c_int), ("rank", C.c_int), ("pinv_eps", C.c_double),
                ("tol", C.c_double), ("maxit", C.c_int), ("stop_on_increase", C.c_int), ("rank_tol", C.c_double),
                ("coeff_rank", C.c_int), ("rank_start", C.c_int), ("rank_step", C.c_int), ("disc", C.c_int),
                ("sketch_over", C.c_int), ("sketch_seed", C.c_uint), ("sketch_keep", C.c_int)]


class lrfg_result(C.Structure):
    _fields_ = [("Aeff", C.c_double), ("iters", C.c_int), ("rel_resid", C.c_double), ("converged", C.c_int),
                ("applies", C.c_int), ("ranks", C.c_int * 4), ("seconds", C.c_double)]


class lrfg_batch_report(C.Structure):
    _fields_ = [("queue_s", C.c_double), ("run_s", C.c_double), ("total_s", C.c_double),
                ("peak_bytes", C.c_double), ("worker", C.c_int), ("group", C.c_int), ("message", C.c_char * 200)]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_ST = C.c_int

# name -> (restype, argtypes); the same set the header declares
SIGNATURES = {
    "lrfg_create": (_ST, [C.POINTER(_P), _I, _P, C.c_size_t]),
    "lrfg_destroy": (_ST, [_P]),
    "lrfg_strerror": (C.c_char_p, [_ST]),
    "lrfg_last_error": (C.c_char_p, [_P]),
    "lrfg_sync": (_ST, [_P]),
    "lrfg_launch_count": (C.c_longlong, [_P]),
    "lrfg_pool_bytes": (_ST, [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "lrfg_profile_classes": (_I, []),
    "lrfg_profile_class_name": (C.c_char_p, [_I]),
    "lrfg_profile_enable": (_ST, [_P, _I]),
    "lrfg_profile_reset": (_ST, [_P]),
    "lrfg_profile_read": (_ST, [_P, _I, C.POINTER(C.c_longlong), C.POINTER(_D), C.POINTER(_D), C.POINTER(_D)]),
    "lrfg_fft_fibres": (_ST, [_P, _P, _P, _I, _I, _I, _I]),
    "lrfg_fft_fibres_f32": (_ST, [_P, _P, _P, _I, _I, _I, _I]),
    "lrfg_fibre_operator": (_ST, [_P, _P, _P, _I, _I, _I, _I, _D, _D]),
    "lrfg_tt_hadamard": (_ST, [_P, C.POINTER(lrfg_tt), C.POINTER(lrfg_tt), C.POINTER(lrfg_tt)]),
    "lrfg_tucker_round": (_ST, [_P, C.POINTER(lrfg_tucker), _I, C.POINTER(lrfg_tucker)]),
    "lrfg_tucker_round_tol": (_ST, [_P, C.POINTER(lrfg_tucker), _I, _D, C.POINTER(lrfg_tucker)]),
    "lrfg_field_from_tucker": (_ST, [_P, C.POINTER(lrfg_tucker), _I, C.POINTER(_P)]),
    "lrfg_tt_add": (_ST, [_P, _D, C.POINTER(lrfg_tt), _D, C.POINTER(lrfg_tt), C.POINTER(lrfg_tt)]),
    "lrfg_tt_round": (_ST, [_P, C.POINTER(lrfg_tt), _I, C.POINTER(lrfg_tt)]),
    "lrfg_tt_round_tol": (_ST, [_P, C.POINTER(lrfg_tt), _I, _D, C.POINTER(lrfg_tt)]),
    "lrfg_tt_round_sketch": (_ST, [_P, C.POINTER(lrfg_tt), _I, C.c_ulonglong, _I, _D, C.POINTER(lrfg_tt)]),
    "lrfg_tt_hadamard_round_sketch": (_ST, [_P, C.POINTER(lrfg_tt), C.POINTER(lrfg_tt), _I, C.c_ulonglong, _I, _D,
                                            C.POINTER(lrfg_tt)]),
    "lrfg_probe_fp64": (_ST, [_P, C.POINTER(_D), C.POINTER(_D)]),
    "lrfg_sym_eig": (_ST, [_P, _P, C.c_int, C.c_int, C.c_int, _P, _P]),
    "lrfg_tt_dot": (_ST, [_P, C.POINTER(lrfg_tt), C.POINTER(lrfg_tt), C.POINTER(_D)]),
    "lrfg_tt_dot_noalloc": (_ST, [_P, C.POINTER(lrfg_tt), C.POINTER(lrfg_tt), _P]),
    "lrfg_tt_precond": (_ST, [_P, C.POINTER(lrfg_tt), _D, _I, C.POINTER(lrfg_tt)]),
    "lrfg_tt_compress": (_ST, [_P, _I, C.POINTER(_I), _P, _I, _D, C.POINTER(lrfg_tt)]),
    "lrfg_tt_expand": (_ST, [_P, C.POINTER(lrfg_tt), _P]),
    "lrfg_problem_create": (_ST, [_P, C.POINTER(lrfg_coeff), C.POINTER(lrfg_opts), C.POINTER(_P)]),
    "lrfg_problem_free": (_ST, [_P]),
    "lrfg_problem_coeff_ranks": (_ST, [_P, C.POINTER(_I)]),
    "lrfg_problem_apply": (_ST, [_P, _P, C.POINTER(_P)]),
    "lrfg_problem_apply_into": (_ST, [_P, _P, _P]),
    "lrfg_problem_rhs": (_ST, [_P, C.POINTER(_D), C.POINTER(_P)]),
    "lrfg_problem_solve": (_ST, [_P, C.POINTER(_D), C.POINTER(lrfg_result), C.POINTER(_P)]),
    "lrfg_problem_aeff": (_ST, [_P, C.POINTER(_D), _P, C.POINTER(_D)]),
    "lrfg_problem_solve_many": (_ST, [_P, _I, C.POINTER(_D), C.POINTER(lrfg_result)]),
    "lrfg_problem_aeff_tensor": (_ST, [_P, C.POINTER(_D), C.POINTER(lrfg_result)]),
    "lrfg_problems_solve": (_ST, [_I, C.POINTER(_P), C.POINTER(_D), C.POINTER(lrfg_result)]),
    "lrfg_solve": (_ST, [_P, C.POINTER(lrfg_coeff), C.POINTER(_D), C.POINTER(lrfg_opts), C.POINTER(lrfg_result),
                         C.POINTER(_P)]),
    "lrfg_field_from_full": (_ST, [_P, _I, C.POINTER(_I), _P, _I, C.POINTER(_P)]),
    "lrfg_field_from_tt": (_ST, [_P, C.POINTER(lrfg_tt), _I, C.POINTER(_P)]),
    "lrfg_field_info": (_ST, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(_I), C.POINTER(_I)]),
    "lrfg_field_export_full": (_ST, [_P, _P, _P, _I]),
    "lrfg_field_export_tt": (_ST, [_P, _P, C.POINTER(_P), _I]),
    "lrfg_field_free": (_ST, [_P]),
    "lrfg_batch_create": (_ST, [C.POINTER(_P), _I, _I, C.c_size_t]),
    "lrfg_batch_submit": (_ST, [_P, C.POINTER(lrfg_coeff), C.POINTER(_D), C.POINTER(lrfg_opts),
                                C.POINTER(C.c_ulonglong)]),
    "lrfg_batch_poll": (_ST, [_P, C.c_ulonglong, _I, C.POINTER(_I), C.POINTER(_ST), C.POINTER(lrfg_result),
                              C.POINTER(lrfg_batch_report)]),
    "lrfg_batch_info": (_ST, [_P, C.POINTER(_I), C.POINTER(_I), C.POINTER(C.c_size_t)]),
    "lrfg_batch_set_group": (_ST, [_P, _I]),
    "lrfg_batch_destroy": (_ST, [_P]),
}

_lib = None


def load(path: str | None = None):
    """Load liblrfg.so (no fallback: a missing library is an error)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"liblrfg.so not found at {p}; build it with `python -m paper_1902_07455_gb300.build`")
    lib = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
