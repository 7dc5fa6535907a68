"""ctypes declarations of libhdcr's C ABI (include/hdcr.h).

Argument marshalling only: every computation runs in the CUDA library.  The
library is loaded from ``paper_1611_06944_gb300/lib/libhdcr.so``; if it is
missing the import fails with an error that says how to build it (there is no
CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "lib", "libhdcr.so")

HDCR_OK = 0
HDCR_C128 = 0
HDCR_C64 = 1
HDCR_C64_FAST = 2
HDCR_C128_TC = 4
HDCR_TIMER_C128_CHEB = 100
HDCR_H16 = 3

STATUS_NAMES = {
    0: "OK", -1: "BAD_ARG", -2: "BAD_GEOMETRY", -3: "NOT_CONVERGED", -4: "NONFINITE",
    -5: "RANK_DEFICIENT", -6: "CUDA", -7: "TIMEOUT", -8: "NO_MEMORY",
}


class hdcr_geom(C.Structure):
    _fields_ = [("L", C.c_int * 4), ("Ls", C.c_int), ("bc_t", C.c_int)]


class hdcr_dwf_params(C.Structure):
    _fields_ = [("M5", C.c_double), ("mf", C.c_double)]


class hdcr_solve_stats(C.Structure):
    _fields_ = [
        ("status", C.c_int), ("iters", C.c_int), ("fine_matvecs", C.c_int),
        ("fine_matvecs_lo", C.c_int), ("coarse_matvecs", C.c_int), ("restarts", C.c_int),
        ("true_resid", C.c_double), ("t_total", C.c_double), ("t_smoother", C.c_double),
        ("t_coarse", C.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


HDCR_SUBSPACE_CR_SMOOTH = 0
HDCR_SUBSPACE_CHEBYSHEV = 1
HDCR_SMOOTHER_CR = 0
HDCR_SMOOTHER_CHEBYSHEV = 1
HDCR_COARSE_CR = 0
HDCR_COARSE_DENSE = 1
HDCR_COARSE_RECURSIVE = 2
HDCR_CYCLE_SYMMETRIC = 0
HDCR_CYCLE_POST = 1


class hdcr_level2_params(C.Structure):
    _fields_ = [("nvec2", C.c_int), ("block", C.c_int * 4), ("smooth_iters", C.c_int), ("cycle_smooth", C.c_int)]


class hdcr_cf_params(C.Structure):
    _fields_ = [("ncomp", C.c_int), ("beta", C.c_double * 15), ("R", C.c_double)]


class hdcr_subspace_params(C.Structure):
    _fields_ = [
        ("nvec", C.c_int), ("block", C.c_int * 4), ("kind", C.c_int), ("order", C.c_int),
        ("lam_cut", C.c_double), ("lam_max", C.c_double), ("filter_dtype", C.c_int),
        ("store_dtype", C.c_int),
    ]


class hdcr_solve_params(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("max_outer", C.c_int), ("restart", C.c_int),
        ("smoother_kind", C.c_int), ("smoother_order", C.c_int), ("cheb_lo", C.c_double),
        ("cheb_hi", C.c_double), ("coarse_solver", C.c_int), ("coarse_tol", C.c_double),
        ("coarse_max", C.c_int), ("inner_dtype", C.c_int), ("cycle", C.c_int),
    ]


_P = C.c_void_p
_I = C.c_int
_D = C.c_double
_SZ = C.c_size_t
_G = C.POINTER(hdcr_geom)
_DP = C.POINTER(hdcr_dwf_params)
_ST = C.POINTER(hdcr_solve_stats)

# name -> (restype, argtypes); every symbol declared in include/hdcr.h
SIGNATURES = {
    "hdcr_strerror": (C.c_char_p, [_I]),
    "hdcr_last_error": (C.c_char_p, []),
    "hdcr_version": (_I, []),
    "hdcr_launch_count": (C.c_ulonglong, []),
    "hdcr_stencil_timer": (_I, [_I]),
    "hdcr_stencil_timer_read": (_I, [_I, C.POINTER(C.c_double), C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "hdcr_stencil_timer_count": (_I, [_I, C.POINTER(C.c_longlong), C.POINTER(C.c_longlong)]),
    "hdcr_probe_fma_rate": (_I, [_I, C.POINTER(C.c_double), _P]),
    "hdcr_tc_gemm_info": (_I, [C.POINTER(C.c_ulonglong), C.POINTER(C.c_ulonglong)]),
    "hdcr_apply_g5dwf": (_I, [_G, _DP, _P, _P, _P, _I, _I, _P]),
    "hdcr_stencil_tune": (_I, [_I, _I]),
    "hdcr_mobius_to_shamir": (_I, [_DP, _D, _P, _P, _I, _SZ, _DP, _P]),
    "hdcr_fermion_encode_h16": (_I, [_G, _P, _I, _P, _I, _P]),
    "hdcr_fermion_decode_h16": (_I, [_G, _P, _P, _I, _I, _P]),
    "hdcr_stencil_tune_info": (_I, [_G, _I, C.POINTER(C.c_int), C.POINTER(C.c_float), _I]),
    "hdcr_apply_gamma5_r5": (_I, [_G, _P, _P, _I, _I, _P]),
    "hdcr_fermion_pack": (_I, [_G, _P, _P, _I, _I, _P]),
    "hdcr_fermion_unpack": (_I, [_G, _P, _P, _I, _I, _P]),
    "hdcr_convert": (_I, [_P, _I, _P, _I, _SZ, _P]),
    "hdcr_cdot": (_I, [_P, _P, _SZ, _I, _P, _P]),
    "hdcr_norm2": (_I, [_P, _SZ, _I, _P, _P]),
    "hdcr_cdot_noalloc": (_I, [_P, _P, _SZ, _I, _P, _P]),
    "hdcr_cr_solve": (_I, [_G, _DP, _P, _P, _P, _I, _D, _I, _ST, _P]),
    "hdcr_cgne_rb_solve": (_I, [_G, _DP, _P, _P, _P, _D, _I, _ST, _P]),
    "hdcr_build_subspace": (_I, [_G, _DP, _P, _P, C.POINTER(hdcr_subspace_params), _P, C.POINTER(_P)]),
    "hdcr_subspace_from_vectors": (_I, [_G, C.POINTER(C.c_int), _I, _P, _I, _P, C.POINTER(_P)]),
    "hdcr_subspace_info": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "hdcr_subspace_get_vectors": (_I, [_P, _P, _P]),
    "hdcr_subspace_destroy": (None, [_P]),
    "hdcr_restrict": (_I, [_P, _P, _P, _I, _I, _P]),
    "hdcr_prolong": (_I, [_P, _P, _P, _I, _I, _P]),
    "hdcr_build_coarse_op": (_I, [_P, _DP, _P, _I, _P, C.POINTER(_P)]),
    "hdcr_coarse_get_op": (_I, [_P, _P, _P]),
    "hdcr_apply_coarse": (_I, [_P, _P, _P, _I, _I, _P]),
    "hdcr_coarse_invert": (_I, [_P, _P]),
    "hdcr_coarse_solve_dense": (_I, [_P, _P, _P, _I, _P]),
    "hdcr_coarse_destroy": (None, [_P]),
    "hdcr_coarse_build_level2": (_I, [_P, C.POINTER(hdcr_level2_params), _P, _P]),
    "hdcr_coarse_level2_info": (_I, [_P, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "hdcr_coarse_level2_get": (_I, [_P, _P, _P, _P]),
    "hdcr_coarse_solve_level2": (_I, [_P, _P, _P, _D, _I, C.POINTER(C.c_int), _P]),
    "hdcr_solve": (_I, [_P, _P, _P, _P, C.POINTER(hdcr_solve_params), _ST, _P]),
    "hdcr_solve_multi": (_I, [_P, _P, _P, _P, _I, C.POINTER(hdcr_solve_params), _I, _ST, _P]),
    "hdcr_apply_cf_overlap": (_I, [_G, _D, C.POINTER(hdcr_cf_params), _P, _P, _P, _I, _I, _P]),
    "hdcr_cf_cr_solve": (_I, [_G, _D, C.POINTER(hdcr_cf_params), _P, _P, _P, _I, _D, _I, _ST, _P]),
    "hdcr_cf_filter": (_I, [_G, _D, C.POINTER(hdcr_cf_params), _P, _P, _I, C.POINTER(hdcr_subspace_params), _P]),
    "hdcr_cf_build_coarse_op": (_I, [_P, _D, C.POINTER(hdcr_cf_params), _P, _P, C.POINTER(_P)]),
    "hdcr_gamma5_split": (_I, [_G, _P, _P, _P, _I, _I, _P]),
    "hdcr_gauge_force": (_I, [_G, _P, _P, _P, _I, _P]),
    "hdcr_gauge_grad": (_I, [_G, _P, _P, _P, _I, _P]),
}


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(
            f"libhdcr.so not found at {path}; build it with "
            "`python -m paper_1611_06944_gb300.build` (needs nvcc). There is no CPU fallback.")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib
