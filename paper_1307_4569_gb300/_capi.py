"""ctypes declarations of libdgt.so (include/dgt.h).  Argument marshalling only.

The library is built in-tree by ``paper_1307_4569_gb300.build``; importing this module
loads it and raises if it is missing -- there is no fallback implementation.
"""
from __future__ import annotations

import ctypes as C
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
# DGT_DEBUG=1 selects the guard-zone bounds-checking build (build.build(debug=True))
LIB_PATH = os.path.join(HERE, "lib", "libdgt_debug.so" if os.environ.get("DGT_DEBUG") == "1" else "libdgt.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "dgt.h")

DGT_OK, DGT_ERR_ARG, DGT_ERR_LENGTH, DGT_ERR_NOT_FRAME, DGT_ERR_CUDA, DGT_ERR_OOM, DGT_ERR_TIMEOUT, \
    DGT_ERR_UNSUPPORTED = range(8)
ROUTE_AUTO, ROUTE_COSET, ROUTE_SHEAR, ROUTE_FIR = range(4)
F32, F64 = 0, 1
WINDOW_FULL, WINDOW_FIR = 0, 1
SYN_ADJOINT, SYN_DUAL, SYN_TIGHT = 0, 1, 2


class Window(C.Structure):
    _fields_ = [("kind", C.c_int), ("len", C.c_int64), ("center", C.c_int64),
                ("data", C.POINTER(C.c_double)), ("is_real", C.c_int)]


class PlanInfo(C.Structure):
    _fields_ = [(n, C.c_int64) for n in ("L", "a", "M", "lambda1", "lambda2", "b", "N", "s")] + \
               [("route", C.c_int), ("precision", C.c_int)] + \
               [(n, C.c_int64) for n in ("s0", "s1", "b_r", "sep_a", "sep_M", "c", "d", "p", "q",
                                         "n_windows", "fir_len", "ola_block", "ola_len")]


class DGTError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (_NAMES.get(status, status), msg))
        self.status = status


_NAMES = {0: "DGT_OK", 1: "DGT_ERR_ARG", 2: "DGT_ERR_LENGTH", 3: "DGT_ERR_NOT_FRAME", 4: "DGT_ERR_CUDA",
          5: "DGT_ERR_OOM", 6: "DGT_ERR_TIMEOUT", 7: "DGT_ERR_UNSUPPORTED"}

_lib = None

vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int
SIGNATURES = {
    "dgt_plan_create": (i32, [C.POINTER(vp), i64, i64, i64, i64, i64, C.POINTER(Window), i32, i32, vp]),
    "dgt_plan_create_ola": (i32, [C.POINTER(vp), i64, i64, i64, i64, i64, C.POINTER(Window), i64, i32, i32, vp]),
    "dgt2_plan_create": (i32, [C.POINTER(vp), i64, i64, i64, i64, i64, C.POINTER(Window),
                               i64, i64, i64, i64, i64, C.POINTER(Window), i32, i32, vp]),
    "dgt2_exec": (i32, [vp, vp, i32, vp, i64, vp]),
    "idgt2_exec": (i32, [vp, vp, vp, i32, i64, i32, vp]),
    "dgt2_plan_status": (i32, [vp, vp]),
    "dgt2_plan_destroy": (None, [vp]),
    "dgt_plan_get_info": (i32, [vp, C.POINTER(PlanInfo)]),
    "dgt_plan_set_window": (i32, [vp, vp, i32, vp]),
    "dgt_exec": (i32, [vp, vp, i32, vp, i64, vp]),
    "dgt_exec_real": (i32, [vp, vp, vp, i64, vp]),
    "idgt_exec_real": (i32, [vp, vp, vp, i64, i32, vp]),
    "idgt_exec": (i32, [vp, vp, vp, i32, i64, i32, vp]),
    "idgt_exec_window": (i32, [vp, vp, vp, i32, i64, vp, i32, vp]),
    "dgt_workspace_bytes": (i32, [vp, i64, C.POINTER(C.c_size_t)]),
    "dgt_exec_ws": (i32, [vp, vp, i32, vp, i64, vp, vp]),
    "idgt_exec_ws": (i32, [vp, vp, vp, i32, i64, i32, vp, vp]),
    "dgt_window_dual": (i32, [vp, vp, vp]),
    "dgt_window_tight": (i32, [vp, vp, vp]),
    "dgt_grad_window": (i32, [vp, vp, i32, vp, vp, i32, i64, vp]),
    "dgt_logmag_loss": (i32, [vp, vp, vp, vp, C.c_double, i64, vp]),
    "dgt_fir_synthesis_noalloc": (i32, [vp, vp, vp, i32, i64, i32, vp]),
    "dgt_plan_bytes": (i32, [vp, C.POINTER(C.c_size_t)]),
    "dgt_sync": (i32, [vp]),
    "dgt_plan_status": (i32, [vp, vp]),
    "dgt_workspace_status": (i32, [vp, vp, vp]),
    "dgt_wait_limit": (C.c_longlong, [C.c_longlong]),
    "dgt_plan_destroy": (None, [vp]),
    "dgt_strerror": (C.c_char_p, [i32]),
    "dgt_last_error": (C.c_char_p, []),
    "dgt_fft_selftest": (i32, [i64, i32, i32, vp, vp, i64, vp]),
    "dgt_fma_rate": (i32, [i32, C.POINTER(C.c_double), vp]),
    "dgt_exec_host": (i32, [vp, vp, i32, vp, i64, i64, vp]),
    "idgt_exec_host": (i32, [vp, vp, vp, i32, i64, i32, i64, vp]),
    "dgt_debug_build": (i32, []),
    "dgt_chirp_table_cap": (C.c_longlong, [C.c_longlong]),
    "dgt_debug_status": (i32, [C.POINTER(C.c_ulonglong), C.POINTER(C.c_longlong), C.c_char_p, C.c_size_t]),
    "dgt_debug_touch_guard": (i32, [vp]),
    "dgt_profile_start": (i32, []),
    "dgt_profile_stop": (i32, [C.c_char_p, C.c_size_t]),
}


def header_functions() -> list[str]:
    """Names of the functions declared in include/dgt.h."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b((?:i?dgt)_[a-z0-9_]+)\s*\(", txt)))


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libdgt.so is not built (%s); run paper_1307_4569_gb300.build.build()" % LIB_PATH)
        h = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def check(status: int) -> None:
    if status != DGT_OK:
        msg = lib().dgt_last_error()
        raise DGTError(status, msg.decode() if msg else "")
