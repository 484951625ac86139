"""ctypes mirror of include/pdlp.h: the structs, the codes and the calls.

Argument marshalling only.  Every array may be a numpy array (host memory) or
a torch tensor (host or CUDA memory); the library copies through unified
virtual addressing either way.  The shared library is loaded from the
package's _build/ directory; if it is missing the import fails (there is no
CPU fallback).
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libpdlp_gb300.so")

PDLP_OK = 0
PDLP_ERR_INVALID_ARG = -1
PDLP_ERR_CUDA = -2
PDLP_ERR_OOM = -3
PDLP_ERR_TIMEOUT = -4
PDLP_ERR_STATE = -5

PDLP_RUNNING, PDLP_OPTIMAL, PDLP_ITER_LIMIT, PDLP_KKT_PASS_LIMIT, PDLP_TIME_LIMIT, PDLP_NUMERICAL_ERROR = range(6)
PDLP_PRIMAL_INFEASIBLE, PDLP_DUAL_INFEASIBLE = 7, 8
STATUS_NAMES = {0: "RUNNING", 1: "OPTIMAL", 2: "ITER_LIMIT", 3: "KKT_PASS_LIMIT", 4: "TIME_LIMIT",
                5: "NUMERICAL_ERROR", 7: "PRIMAL_INFEASIBLE", 8: "DUAL_INFEASIBLE"}

PDLP_FP64, PDLP_FP32, PDLP_FP32_REFINE = 0, 1, 2


class pdlp_csr(C.Structure):
    _fields_ = [("m", C.c_int32), ("n", C.c_int32), ("nnz", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p)]


class pdlp_options(C.Structure):
    _fields_ = [("rel_tol", C.c_double), ("iter_limit", C.c_int64), ("kkt_pass_limit", C.c_int64),
                ("time_limit_s", C.c_double), ("precision", C.c_int32), ("ruiz_iters", C.c_int32),
                ("pock_chambolle", C.c_int32), ("eval_every", C.c_int32),
                ("adaptive_restart", C.c_int32), ("pw_update", C.c_int32),
                ("pw_smoothing", C.c_double), ("primal_importance", C.c_double),
                ("beta_suff", C.c_double), ("beta_nec", C.c_double), ("beta_art", C.c_double),
                ("eps_zero", C.c_double), ("inner_tol", C.c_double), ("refine_rounds", C.c_int32),
                ("unroll_T", C.c_int32), ("ckpt_every", C.c_int32), ("use_graph", C.c_int32),
                ("persistent", C.c_int32), ("step_policy", C.c_int32), ("presolve", C.c_int32),
                ("omega0", C.c_double),
                ("restart_to_current", C.c_int32), ("wait_limit_us", C.c_int32), ("mp_breaking", C.c_double),
                ("mp_downscaling", C.c_double), ("mp_interpolation", C.c_double), ("stream", C.c_void_p)]


class pdlp_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("returned_average", C.c_int32), ("iters", C.c_int64),
                ("kkt_passes", C.c_int64), ("restarts", C.c_int64), ("refine_rounds", C.c_int32),
                ("engine", C.c_int32), ("primal_obj", C.c_double), ("dual_obj", C.c_double),
                ("gap", C.c_double), ("pres", C.c_double), ("dres", C.c_double),
                ("rel_gap", C.c_double), ("rel_pres", C.c_double), ("rel_dres", C.c_double),
                ("seconds", C.c_double), ("step_size", C.c_double), ("primal_weight", C.c_double),
                ("finish_iters", C.c_int64)]

    def asdict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_ }
        d["status_name"] = STATUS_NAMES.get(self.status, str(self.status))
        d["rel_kkt"] = max(self.rel_gap, self.rel_pres, self.rel_dres)
        return d


P = C.c_void_p
_SIGNATURES = {
    "pdlp_default_options": ([C.POINTER(pdlp_options)], C.c_int),
    "pdlp_create": ([C.POINTER(pdlp_csr), P, P, P, P, P, C.POINTER(pdlp_options), C.POINTER(P)], C.c_int),
    "pdlp_solve": ([P, P, P, P, P, C.POINTER(pdlp_result)], C.c_int),
    "pdlp_unroll": ([P, C.c_int32, C.c_int32, P, P, P, P, P], C.c_int),
    "pdlp_grad": ([P, P, P, P, P, P], C.c_int),
    "pdlp_get_scaled": ([P] + [P] * 11, C.c_int),
    "pdlp_normalized_gap": ([P, P, P, C.c_double, C.c_double, P, P], C.c_int),
    "pdlp_solve_batch": ([C.c_int32] + [P] * 13 + [C.POINTER(pdlp_options), P, P, P], C.c_int),
    "pdlp_batch_lanes": ([C.c_int32, P, P, C.c_int32], C.c_int),
    "pdlp_get_trace": ([P, P, C.c_int32, C.POINTER(C.c_int32)], C.c_int),
    "pdlp_time_step_kernels": ([P, C.c_int32, P], C.c_int),
    "pdlp_normalized_gap_noalloc": ([C.c_int32, C.c_int32] + [P] * 7 + [C.c_double, C.c_double, P, P, P],
                                    C.c_int),
    "pdlp_last_error": ([P], C.c_char_p),
    "pdlp_destroy": ([P], None),
}

_lib = None


def load():
    """Loads libpdlp_gb300.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with paper_2106_04756_gb300.build.build()")
        lib = C.CDLL(LIB_PATH)
        for name, (args, res) in _SIGNATURES.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
    return _lib


class PdlpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"PDLP error {code}: {msg}")
        self.code = code


def check(code: int, ctx=None):
    if code != PDLP_OK:
        msg = load().pdlp_last_error(ctx)
        raise PdlpError(code, msg.decode() if msg else "")
    return code
