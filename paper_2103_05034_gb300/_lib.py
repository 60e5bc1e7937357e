"""ctypes loader for libdwfmg.so (the C ABI declared in include/dwfmg.h).

Loading fails loudly: there is no CPU fallback anywhere in this package.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdwfmg.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dwfmg.h")

_lib = None

DWF_OK, DWF_EINVAL, DWF_ENOMEM, DWF_ENOCONV, DWF_ENAN, DWF_ECUDA, DWF_ETIMEOUT, DWF_ERANGE = \
    0, -1, -2, -3, -4, -5, -6, -7
F64, F32, F16S, TF32 = 0, 1, 2, 3
SOLVE_F64, SOLVE_MIXED_F32, SOLVE_MIXED_F16 = 0, 1, 2
HOP_VARIANTS = 26  # DWF_HOP_VARIANTS
STATUS_NAMES = {0: "DWF_OK", -1: "DWF_EINVAL", -2: "DWF_ENOMEM", -3: "DWF_ENOCONV",
                -4: "DWF_ENAN", -5: "DWF_ECUDA", -6: "DWF_ETIMEOUT", -7: "DWF_ERANGE"}


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("reliable_updates", C.c_int),
                ("coarse_iterations", C.c_int), ("status", C.c_int),
                ("fine_matmuls", C.c_double), ("true_residual", C.c_double),
                ("seconds", C.c_double), ("setup_seconds", C.c_double),
                ("coarse_op_seconds", C.c_double), ("graph_replays", C.c_int), ("pad_", C.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


SUBSPACE_BATCH, SUBSPACE_RECURSIVE = 0, 1
COARSE_CG, COARSE_RB, COARSE_DEFLATED = 0, 1, 2
ARITH_FP64, ARITH_FLOAT_FLOAT = 0, 1


class MGParams(C.Structure):
    _fields_ = [("block", C.c_int * 4), ("nbasis", C.c_int), ("subspace_mode", C.c_int),
                ("mf", C.c_double), ("lambda_lo", C.c_double), ("lambda_max", C.c_double),
                ("filter_order", C.c_int), ("delta", C.c_int), ("smooth_lo", C.c_double),
                ("smooth_hi", C.c_double), ("smooth_order", C.c_int), ("coarse_tol", C.c_double),
                ("coarse_maxiter", C.c_int), ("nkrylov", C.c_int), ("maxiter", C.c_int),
                ("no_graph", C.c_int), ("coarse_solver", C.c_int), ("coarse_nev", C.c_int),
                ("coarse_lanczos", C.c_int), ("coarse_cheb_order", C.c_int), ("coarse_cheb_lo", C.c_double)]


class HybridParams(C.Structure):
    _fields_ = [("block", C.c_int * 4), ("nbasis4", C.c_int), ("mass4", C.c_double),
                ("lambda_lo4", C.c_double), ("lambda_max4", C.c_double), ("order4", C.c_int),
                ("nbasis1", C.c_int), ("lambda_lo1", C.c_double), ("lambda_max1", C.c_double),
                ("order1", C.c_int), ("smooth1_lo", C.c_double), ("smooth1_hi", C.c_double),
                ("smooth1_order", C.c_int), ("kcycle", C.c_int)]


def header_functions():
    """Names of the functions declared in include/dwfmg.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*([a-z_][a-z0-9_]*)\s*\(",
                       txt, flags=re.M)
    return sorted(set(n for n in names if n not in ("if", "defined")))


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(
                f"{LIB_PATH} is missing: build it with "
                "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class DWFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code, ctx=None):
    if code != DWF_OK:
        msg = lib().dwf_last_error(ctx).decode() if ctx else ""
        raise DWFError(code, msg)
    return code


P, I, D, I64 = C.c_void_p, C.c_int, C.c_double, C.c_int64
_SIGS = {
    "dwf_ctx_create": (I, [C.POINTER(P), C.POINTER(C.c_int), I, D, P, P]),
    "dwf_ctx_destroy": (I, [P]),
    "dwf_last_error": (C.c_char_p, [P]),
    "dwf_half_sites": (I64, [P]),
    "dwf_half_bytes": (I64, [P, I]),
    "dwf_counters": (I, [P, C.POINTER(I64), C.POINTER(D)]),
    "dwf_reset_counters": (I, [P]),
    "dwf_autotune": (I, [P, I, I, C.POINTER(D), P]),
    "dwf_set_f64_arithmetic": (I, [P, I]),
    "dwf_get_f64_arithmetic": (I, [P]),
    "dwf_set_hop_variant": (I, [P, I, I]),
    "dwf_get_hop_variant": (I, [P, I]),
    "dwf_dhop": (I, [P, P, P, I, I, I, I, P]),
    "dwf_mooee": (I, [P, P, P, D, I, I, I, P]),
    "dwf_mooee_inv": (I, [P, P, P, D, I, I, I, P]),
    "dwf_mpc": (I, [P, P, P, D, I, I, I, P]),
    "dwf_mpcdag_mpc": (I, [P, P, P, D, I, I, P]),
    "dwf_ddw": (I, [P, P, P, D, I, I, I, P]),
    "dwf_hdw": (I, [P, P, P, D, I, I, P]),
    "dwf_norm2": (I, [P, C.POINTER(D), P, I64, I, P]),
    "dwf_cdot": (I, [P, C.POINTER(D), P, P, I64, I, P]),
    "dwf_norm2_noalloc": (I, [C.POINTER(D), P, I64, I, P]),
    "dwf_selftest_wait_timeout": (I, [C.POINTER(C.c_int), P]),
    "dwf_measure_fma_peaks": (I, [C.POINTER(D), C.POINTER(D), P]),
    "rbcg_solve": (I, [P, P, P, D, D, I, I, C.POINTER(SolveStats), P]),
    "rbcg2_solve": (I, [P, P, P, D, D, I, I, C.POINTER(SolveStats), P]),
    "dwf_power_max": (I, [P, C.POINTER(D), P, D, I, I, P]),
    "dwf_force": (I, [P, P, P, C.POINTER(D), I, I, P]),
    "dwf_ratio_force": (I, [P, P, P, P, C.POINTER(D), C.POINTER(D), I, I, P]),
    "dwf_pf_action": (I, [P, C.POINTER(D), P, P, C.POINTER(D), I, P]),
    "rbcg_normal_solve": (I, [P, P, P, D, D, I, I, C.POINTER(SolveStats), P]),
    "cgnr_solve": (I, [P, P, P, D, D, I, C.POINTER(SolveStats), P]),
    "rbcg_solve_batch": (I, [P, P, P, C.POINTER(D), I, D, I, I, C.POINTER(SolveStats), P]),
    "rbcg_normal_solve_batch": (I, [P, P, P, C.POINTER(D), I, D, I, I, C.POINTER(SolveStats), P]),
    "cheby_filter": (I, [P, P, P, I, D, D, I, D, I, P]),
    "cheby_recursive_basis": (I, [P, P, P, D, D, I, I, I, D, I, P]),
    "dwf_chiral_project": (I, [P, P, P, I, I, I, P]),
    "block_orthonormalise": (I, [P, P, I, I, C.POINTER(C.c_int), P]),
    "coarse_build": (I, [P, P, I, I, C.POINTER(C.c_int), D, I, C.POINTER(P), P]),
    "coarse_destroy": (I, [P]),
    "coarse_export": (I, [P, P, C.POINTER(C.c_int)]),
    "coarse_apply": (I, [P, P, P, I, I, P]),
    "coarse_apply_status": (I, [P, P]),
    "coarse_solve": (I, [P, P, P, D, I, C.POINTER(C.c_int), P]),
    "coarse_solve_rb": (I, [P, P, P, D, I, C.POINTER(C.c_int), P]),
    "coarse_solve_multi": (I, [P, P, P, I, D, I, C.POINTER(C.c_int), I, P]),
    "coarse_deflate": (I, [P, P, I, I, I, D, D, C.POINTER(D), P]),
    "coarse_export_deflation": (I, [P, P, C.POINTER(D), C.POINTER(C.c_int)]),
    "dwf_restrict": (I, [P, P, P, P, I, C.POINTER(C.c_int), I, I, P]),
    "dwf_prolong": (I, [P, P, P, P, I, C.POINTER(C.c_int), I, I, I, P]),
    "mg_setup": (I, [P, C.POINTER(MGParams), P, C.POINTER(P), P]),
    "mg_destroy": (I, [P]),
    "mg_export_basis": (I, [P, P]),
    "mg_coarse": (P, [P]),
    "mg_smooth": (I, [P, P, P, P]),
    "mg_precondition": (I, [P, P, P, P]),
    "mg_solve": (I, [P, P, P, D, C.POINTER(SolveStats), P]),
    "mg_setup_hybrid": (I, [P, C.POINTER(MGParams), C.POINTER(HybridParams), P, P, C.POINTER(P), P]),
    "mg_hybrid_export": (I, [P, I, P]),
    "mg_hybrid_level1": (I, [P, I, P, P, I, P]),
}

