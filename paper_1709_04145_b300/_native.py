"""ctypes binding of ``libpbad.so`` (argument marshalling only)."""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpbad.so")

_lib = None

PBAD_OK = 0
ERRORS = {-1: "PBAD_ERR_ARG", -2: "PBAD_ERR_CUDA", -3: "PBAD_ERR_ALLOC", -4: "PBAD_ERR_UNSUPPORTED"}

# every symbol the C header declares
SYMBOLS = ("pbad_version", "pbad_last_error", "pbad_colloc", "pbad_model_create",
           "pbad_model_destroy", "pbad_model_info", "pbad_batch_create", "pbad_batch_destroy",
           "pbad_batch_info", "pbad_eval_objective_grad", "pbad_step", "pbad_rollout",
           "pbad_fp64_peak", "pbad_eval_objective_grad_static", "pbad_step_backward",
           "pbad_link_points", "pbad_batch_set_threads", "pbad_model_set_drag",
           "pbad_model_set_contact", "pbad_batch_set_queue", "pbad_batch_set_mapping",
           "pbad_fp64_mma_peak", "pbad_batch_set_precision", "pbad_rollout_backward",
           "pbad_batch_set_bucket_mapping", "pbad_damped_gram_solve",
           "pbad_batch_set_newton_cta_min", "pbad_batch_set_newton_split")


class PBADError(RuntimeError):
    pass


def lib():
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libpbad.so not built ({LIB_PATH}); run __graft_entry__.build() "
                              "or python -m paper_1709_04145_b300._build")
        L = C.CDLL(LIB_PATH)
        vp, dp, ip, i64p = C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int64)
        i32, i64, f64 = C.c_int32, C.c_int64, C.c_double
        L.pbad_version.restype = C.c_int
        L.pbad_last_error.restype = C.c_char_p
        L.pbad_colloc.argtypes = [i32, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.pbad_model_create.argtypes = [i32, C.POINTER(C.c_int32), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_double), i64, C.POINTER(C.c_double),
                                        C.POINTER(C.c_double), C.POINTER(C.c_double), i32,
                                        C.POINTER(C.c_void_p)]
        L.pbad_model_destroy.argtypes = [vp]
        L.pbad_model_info.argtypes = [vp, C.POINTER(C.c_int32), C.POINTER(C.c_int32), i64p]
        L.pbad_batch_create.argtypes = [i32, C.POINTER(C.c_void_p), i32, i32, i32,
                                        C.POINTER(C.c_void_p)]
        L.pbad_batch_destroy.argtypes = [vp]
        L.pbad_batch_info.argtypes = [vp, i64p, i64p, i64p]
        L.pbad_eval_objective_grad.argtypes = [vp, dp, dp, dp, dp, f64, i32, dp, dp, dp, vp]
        L.pbad_step.argtypes = [vp, dp, dp, dp, f64, i32, C.POINTER(C.c_int32), i32, f64, i32,
                                dp, dp, dp, ip, ip, vp]
        L.pbad_rollout.argtypes = [vp, dp, dp, dp, i32, f64, i32, C.POINTER(C.c_int32), i32, f64,
                                   i32, dp, dp, dp, dp, ip, ip, ip, ip, ip, dp, dp, vp]
        L.pbad_rollout_backward.argtypes = [vp, dp, dp, dp, dp, i32, f64, i32, dp, dp, dp, dp, dp,
                                            ip, vp]
        L.pbad_fp64_peak.argtypes = [i32, C.POINTER(C.c_double)]
        L.pbad_fp64_mma_peak.argtypes = [i32, C.POINTER(C.c_double)]
        L.pbad_batch_set_threads.argtypes = [vp, i32]
        L.pbad_batch_set_queue.argtypes = [vp, i32]
        L.pbad_batch_set_mapping.argtypes = [vp, i32]
        L.pbad_batch_set_precision.argtypes = [vp, i32]
        L.pbad_batch_set_bucket_mapping.argtypes = [vp, C.POINTER(C.c_int32)]
        L.pbad_damped_gram_solve.argtypes = [C.c_int64, i32, vp, vp, C.c_double, vp, vp, vp, vp, vp]
        L.pbad_batch_set_newton_cta_min.argtypes = [vp, i32]
        L.pbad_batch_set_newton_split.argtypes = [vp, i32]
        L.pbad_model_set_drag.argtypes = [vp, f64]
        L.pbad_model_set_contact.argtypes = [vp, i32, C.POINTER(C.c_int32), C.POINTER(C.c_double),
                                             f64, f64, f64]
        L.pbad_link_points.argtypes = [vp, dp, C.POINTER(C.c_int32), dp, dp, dp, vp]
        L.pbad_step_backward.argtypes = [vp, dp, dp, dp, dp, dp, f64, i32, dp, dp, dp, ip, vp]
        L.pbad_eval_objective_grad_static.argtypes = [vp, dp, dp, dp, dp, f64, i32, dp, dp, dp, vp]
        for name in SYMBOLS:
            getattr(L, name).restype = C.c_char_p if name == "pbad_last_error" else C.c_int
        _lib = L
    return _lib


def check(rc: int, what: str):
    if rc != PBAD_OK:
        msg = lib().pbad_last_error().decode()
        raise PBADError(f"{what} failed: {ERRORS.get(rc, rc)}: {msg}")
