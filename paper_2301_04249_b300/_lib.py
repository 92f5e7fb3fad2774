"""ctypes declarations of librteom.so (include/rteom.h).  Marshalling only."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librteom.so")

RTEOM_OK = 0
RTEOM_ERR_ARG = -1
RTEOM_ERR_OOM = -2
RTEOM_ERR_CUDA = -3
RTEOM_ERR_NOT_CONVERGED = -4
RTEOM_ERR_NONFINITE = -5
RTEOM_ERR_STATE = -6
RTEOM_FP64 = 0
RTEOM_SPLIT_BF16 = 1
RTEOM_SPLIT_TF32 = 2
RTEOM_FP64_OZAKI = 3
RTEOM_SPLIT_FP16 = 4
RTEOM_FLAG_CUMULANT_NO_FOV = 1
RTEOM_FLAG_LADDER_CHOLESKY = 2
RTEOM_FLAG_ANDERSON = 4
RTEOM_FLAG_GROUPED = 8
RTEOM_REQ_QUEUED = 0
RTEOM_REQ_RUNNING = 1
RTEOM_REQ_DONE = 2
RTEOM_REQ_FAILED = 3
RTEOM_REQ_CANCELLED = 4

_dp = ctypes.POINTER(ctypes.c_double)
_llp = ctypes.POINTER(ctypes.c_longlong)
_vp = ctypes.c_void_p

# name -> (restype, argtypes); every entry point of include/rteom.h
SIGNATURES = {
    "rteom_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    _dp, _dp, _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp]),
    "rteom_propagate": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int, _dp]),
    "rteom_propagate_group": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int,
                                             ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                             ctypes.POINTER(_dp)]),
    "rteom_spectrum": (ctypes.c_int, [_vp, _dp, ctypes.c_int, ctypes.c_double, _dp]),
    "rteom_get_info": (ctypes.c_int, [_vp, _dp, _dp, _llp, _llp]),
    "rteom_state_size": (ctypes.c_longlong, [_vp]),
    "rteom_get_cumulant": (ctypes.c_int, [_vp, ctypes.c_longlong, _dp, _dp]),
    "rteom_get_state": (ctypes.c_int, [_vp, _dp, _llp, _dp]),
    "rteom_set_state": (ctypes.c_int, [_vp, _dp, ctypes.c_longlong, _dp]),
    "rteom_debug_residual": (ctypes.c_int, [_vp, _dp, _dp, _dp]),
    "rteom_debug_residual_sparse": (ctypes.c_int, [_vp, _llp, _dp, ctypes.c_longlong, _llp,
                                                   ctypes.c_longlong, _dp]),
    "rteom_set_timing": (ctypes.c_int, [_vp, ctypes.c_int]),
    "rteom_get_timing": (ctypes.c_int, [_vp, _dp, _llp, _dp, _dp, ctypes.c_int]),
    "rteom_kernel_launches": (ctypes.c_longlong, [_vp]),
    "rteom_server_create": (ctypes.c_int, [ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int,
                                           ctypes.c_int]),
    "rteom_server_submit": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp,
                                           _dp, _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_int, _llp]),
    "rteom_server_submit_sweep": (ctypes.c_int, [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                 _dp, _dp, _dp, _dp,
                                                 ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                                 ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                 ctypes.c_double, ctypes.c_int, _llp]),
    "rteom_server_poll": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int), _dp, _dp]),
    "rteom_server_wait": (ctypes.c_int, [_vp, ctypes.c_longlong, ctypes.c_double]),
    "rteom_server_cancel": (ctypes.c_int, [_vp, ctypes.c_longlong]),
    "rteom_server_stats": (ctypes.c_int, [_vp, _llp, _llp, _llp, _llp, _dp, _dp]),
    "rteom_plan_bytes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_int, _dp]),
    "rteom_server_estimate_bytes": (ctypes.c_double, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                      ctypes.c_int]),
    "rteom_server_destroy": (None, [_vp]),
    "rteom_ecorr_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp,
                                           _vp, _vp, ctypes.c_char_p, ctypes.c_int]),
    "rteom_destroy": (None, [_vp]),
    "rteom_last_error": (ctypes.c_char_p, [_vp]),
}

_lib = None


def load() -> ctypes.CDLL:
    """Load librteom.so from the package directory; raise if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is not built; run `python -m paper_2301_04249_b300.build` "
                          "(the library has no CPU fallback)")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib
