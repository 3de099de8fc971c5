"""ctypes declarations of libssoct's C ABI (include/ssoct.h); marshalling only.

Every function of the header is exposed here under its C name with argtypes and
restype set.  Loading fails loudly (OSError with the reason) when the library
has not been built: there is no fallback implementation.
"""

from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libssoct.so")

SSOCT_OK = 0
SSOCT_EINVAL = 1
SSOCT_ENOMEM = 2
SSOCT_ECUDA = 3
SSOCT_EAGAIN = 4
SSOCT_ENOTREADY = 5
SSOCT_EDROPPED = 6
SSOCT_ETIMEOUT = 7
SSOCT_EUNSUPPORTED = 8
SSOCT_FLAG_MAGNITUDE = 0x1
SSOCT_FLAG_TC_AXIAL = 0x2
SSOCT_FLAG_PUPIL = 0x4
SSOCT_FLAG_AXIAL_FIRST = 0x8

STATUS_NAMES = {
    0: "SSOCT_OK", 1: "SSOCT_EINVAL", 2: "SSOCT_ENOMEM", 3: "SSOCT_ECUDA", 4: "SSOCT_EAGAIN",
    5: "SSOCT_ENOTREADY", 6: "SSOCT_EDROPPED", 7: "SSOCT_ETIMEOUT", 8: "SSOCT_EUNSUPPORTED",
}


class ssoct_window(C.Structure):
    _fields_ = [("x0", C.c_int), ("y0", C.c_int), ("wx", C.c_int), ("wy", C.c_int)]


class ssoct_plan_info_t(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("nlambda", C.c_int),
        ("window", ssoct_window),
        ("lambda1_m", C.c_double),
        ("dprime_x_m", C.c_double), ("dprime_y_m", C.c_double),
        ("z_b_m", C.c_double),
        ("aliased_chirp", C.c_int),
        ("prefactor_re", C.c_double), ("prefactor_im", C.c_double),
        ("workspace_bytes", C.c_size_t),
        ("ring_slots", C.c_int),
    ]


class ssoct_tune_t(C.Structure):
    _fields_ = [("lag", C.c_int), ("ring_slots", C.c_int), ("tc_axial", C.c_int), ("ms", C.c_double),
                ("from_cache", C.c_int), ("candidates", C.c_int), ("axial_first", C.c_int)]


ssoct_plan = C.c_void_p

# name -> (restype, argtypes); mirrors include/ssoct.h
SIGNATURES = {
    "ssoct_create_plan": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                    C.POINTER(C.c_double), C.POINTER(ssoct_window), C.c_uint,
                                    C.POINTER(ssoct_plan)]),
    "ssoct_plan_info": (C.c_int, [ssoct_plan, C.POINTER(ssoct_plan_info_t)]),
    "ssoct_workspace_size": (C.c_int, [ssoct_plan, C.POINTER(C.c_size_t)]),
    "ssoct_workspace_bytes": (C.c_int, [ssoct_plan, C.POINTER(C.c_size_t)]),
    "ssoct_set_workspace": (C.c_int, [ssoct_plan, C.c_void_p, C.c_size_t]),
    "ssoct_push_frames": (C.c_int, [ssoct_plan, C.c_void_p, C.c_int, C.c_int, C.c_int64, C.c_void_p]),
    "ssoct_reconstruct_volume": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssoct_reconstruct_frames": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssoct_reconstruct_sliding": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssoct_reconstruct_frames_noalloc": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssoct_get_cuts": (C.c_int, [ssoct_plan, C.c_void_p, C.c_int, C.c_int, C.c_int,
                                 C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "ssoct_sync": (C.c_int, [ssoct_plan, C.c_void_p]),
    "ssoct_sliding_cuts": (C.c_int, [ssoct_plan, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                     C.c_void_p]),
    "ssoct_set_pupil": (C.c_int, [ssoct_plan, C.POINTER(C.c_double), C.c_int, C.c_double]),
    "ssoct_sharpness": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "ssoct_inject_stall": (C.c_int, [ssoct_plan, C.c_uint, C.c_ulonglong]),
    "ssoct_profile": (C.c_int, [ssoct_plan, C.c_int]),
    "ssoct_profile_read": (C.c_int, [ssoct_plan, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_int)]),
    "ssoct_last_error": (C.c_char_p, [ssoct_plan]),
    "ssoct_status_string": (C.c_char_p, [C.c_int]),
    "ssoct_destroy_plan": (None, [ssoct_plan]),
    "ssoct_autotune": (C.c_int, [ssoct_plan, C.c_void_p, C.c_void_p, C.c_char_p, C.c_void_p,
                                 C.POINTER(ssoct_tune_t)]),
    "ssoct_batch_create": (C.c_int, [C.POINTER(ssoct_plan), C.c_int, C.c_int, C.POINTER(C.c_void_p)]),
    "ssoct_batch_run": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_void_p]),
    "ssoct_batch_sync": (C.c_int, [C.c_void_p, C.c_void_p]),
    "ssoct_batch_captures": (C.c_int, [C.c_void_p]),
    "ssoct_batch_last_error": (C.c_char_p, [C.c_void_p]),
    "ssoct_batch_destroy": (None, [C.c_void_p]),
}

_lib = None


def lib() -> C.CDLL:
    """The loaded library (built in-tree by paper_2003_08960_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise OSError(f"libssoct.so is not built at {LIB_PATH}; run paper_2003_08960_gb300.build.build() "
                          "(needs nvcc). There is no CPU fallback.")
        l = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib
