"""ctypes declarations of the C ABI in include/madflow_gb300.h.

Loading fails loudly when the CUDA library has not been built: there is no
CPU fallback for any call.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libmadflow_gb300.so")

MF_EE_MUMU, MF_GG_TT, MF_UU_TT, MF_GG_TTG, MF_UG_TTU, MF_GG_TTGG, MF_GG_TTGGG = 0, 1, 2, 3, 4, 5, 6
MF_FP64, MF_MIXED = 0, 1
STATUS = {0: "MF_OK", 1: "MF_ERR_ARG", 2: "MF_ERR_CUDA", 3: "MF_ERR_TIMEOUT", 4: "MF_ERR_NUMERIC",
          5: "MF_ERR_UNSUPPORTED"}


class MfConfig(C.Structure):
    _fields_ = [("mt", C.c_double), ("alpha_s", C.c_double), ("mz", C.c_double), ("wz", C.c_double),
                ("alpha_em_inv", C.c_double), ("gf", C.c_double), ("pt_min", C.c_double),
                ("eta_max", C.c_double), ("dr_min", C.c_double), ("seed", C.c_ulonglong),
                ("channel", C.c_uint), ("n_bins", C.c_int), ("alpha", C.c_double), ("precision", C.c_int)]


class MfResult(C.Structure):
    _fields_ = [("sigma_pb", C.c_double), ("error_pb", C.c_double), ("chi2_dof", C.c_double),
                ("n_events_total", C.c_longlong), ("n_pass", C.c_longlong), ("n_nan", C.c_longlong),
                ("n_iter", C.c_int), ("dsigma_dmt", C.c_double), ("dsigma_dmt_error", C.c_double),
                ("dsigma_dalphas", C.c_double)]


class MfCuts(C.Structure):
    _fields_ = [("pt_min", C.c_double), ("eta_max", C.c_double), ("dr_min", C.c_double)]


class MfObs(C.Structure):
    _fields_ = [("n_bins", C.c_int), ("lo", C.c_double), ("hi", C.c_double)]


class MfEventArrays(C.Structure):
    _fields_ = [("u", C.c_void_p), ("x", C.c_void_p), ("bins", C.c_void_p), ("w", C.c_void_p),
                ("mask", C.c_void_p), ("me2", C.c_void_p), ("momenta", C.c_void_p)]


class MfError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library {LIB_PATH} is not built; run __graft_entry__.build() "
                               "(there is no CPU fallback)")
        L = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_longlong
        sig = {
            "mf_default_config": (C.c_int, [C.POINTER(MfConfig)]),
            "mf_process_info": (C.c_int, [C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
            "mf_create": (C.c_int, [C.POINTER(vp), C.POINTER(MfConfig), dp, C.c_int, C.c_int, C.c_int,
                                    C.c_double, C.c_double, C.c_double, vp]),
            "mf_destroy": (None, [vp]),
            "mf_last_error": (C.c_char_p, [vp]),
            "mf_set_precision": (C.c_int, [vp, C.c_int]),
            "mf_set_pdf": (C.c_int, [vp, dp]),
            "mf_set_schedule": (C.c_int, [vp, C.c_int]),
            "mf_set_helicity_split": (C.c_int, [vp, C.c_int]),
            "mf_set_helicity_sampling": (C.c_int, [vp, C.c_int, C.c_uint]),
            "mf_set_observable": (C.c_int, [vp, C.POINTER(MfObs)]),
            "mf_get_observable": (C.c_int, [vp, dp, dp, dp]),
            "mf_device_status": (C.c_int, [vp]),
            "mf_selftest_wait": (C.c_int, [vp, C.c_uint]),
            "mf_integrate": (C.c_int, [vp, C.c_int, C.c_double, C.POINTER(MfCuts), i64, C.c_int, C.c_int,
                                       C.POINTER(MfResult), dp, dp]),
            "mf_integrate_grid": (C.c_int, [vp, C.c_int, C.c_double, C.POINTER(MfCuts), i64, C.c_int, C.c_uint, dp,
                                            C.c_int, C.POINTER(MfResult), dp, dp]),
            "mf_vegas_pass": (C.c_int, [vp, C.c_int, C.c_double, vp, i64, i64, C.c_uint, vp, vp,
                                        C.POINTER(MfEventArrays)]),
            "mf_vegas_refine": (C.c_int, [vp, C.c_int, C.c_int, C.c_double, vp, vp]),
            "mf_evaluate": (C.c_int, [vp, C.c_int, vp, i64, vp, vp]),
            "mf_helicity_profile": (C.c_int, [vp, C.c_int, vp, i64, vp]),
            "mf_set_couplings": (C.c_int, [vp, C.c_double, C.c_double]),
            "mf_vegas_pass_grad": (C.c_int, [vp, C.c_int, C.c_double, vp, i64, i64, C.c_uint, vp, vp]),
            "mf_vegas_pass_static": (C.c_int, [C.c_int, C.POINTER(MfConfig), C.c_double, vp, C.c_int, C.c_int, C.c_int,
                                               C.c_double, C.c_double, C.c_double, vp, i64, i64, C.c_uint, vp, vp]),
            "mf_integrate_batch": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(i64), C.c_double,
                                             C.POINTER(MfCuts), C.c_int, C.c_int, C.POINTER(MfResult),
                                             C.POINTER(MfResult), dp]),
            "mf_batch_grad": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(i64), C.c_double,
                                        C.POINTER(MfCuts), C.c_uint, dp]),
            "mf_batch_pass": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(i64), C.c_double, vp, C.c_uint,
                                        vp, C.POINTER(MfEventArrays)]),
            "mf_set_batch_schedule": (C.c_int, [vp, C.c_int, C.c_int, i64, i64, C.c_int, C.c_int]),
            "mf_autotune_batch": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int), C.POINTER(i64), C.c_double,
                                            C.POINTER(C.c_int)]),
            "mf_measure_fma_peak": (C.c_int, [C.c_int, vp, dp]),
            "mf_selftest_df": (C.c_int, [C.c_int, vp, i64, vp, vp]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return ["mf_default_config", "mf_process_info", "mf_create", "mf_destroy", "mf_last_error",
            "mf_set_precision", "mf_set_pdf", "mf_set_schedule", "mf_set_helicity_split", "mf_set_helicity_sampling", "mf_set_observable", "mf_get_observable", "mf_device_status", "mf_selftest_wait", "mf_integrate", "mf_integrate_grid", "mf_vegas_pass", "mf_vegas_refine", "mf_evaluate", "mf_helicity_profile",
            "mf_vegas_pass_static", "mf_set_couplings", "mf_vegas_pass_grad",
            "mf_integrate_batch", "mf_batch_pass", "mf_batch_grad", "mf_set_batch_schedule", "mf_autotune_batch",
            "mf_measure_fma_peak", "mf_selftest_df"]
