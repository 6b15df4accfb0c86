"""ctypes binding of libpsolve.so (argument marshalling only).

The library is built in-tree by `paper_1408_6497_gb300.build.build()` (or
`__graft_entry__.build()`).  Nothing here computes: every step of a solve
runs in the CUDA kernels behind the C ABI declared in include/psolve.h.  If
the library is missing, loading fails loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpsolve.so")

F64, F32, F32_TC = 0, 1, 2
DTYPE_CODES = {"f64": F64, "f32": F32, "f32_tc": F32_TC}

STATUS = {0: "PSOLVE_OK", 1: "PSOLVE_ERR_INVALID_ARG", 2: "PSOLVE_ERR_UNSUPPORTED_SIZE",
          3: "PSOLVE_ERR_OOM", 4: "PSOLVE_ERR_CUDA", 5: "PSOLVE_ERR_TIMEOUT", 6: "PSOLVE_ERR_INTERNAL"}

# Every symbol include/psolve.h declares.
EXPORTS = ("psolve_plan_create", "psolve_plan_create_many", "psolve_execute", "psolve_adjoint",
           "psolve_execute_host", "psolve_execute_host_async", "psolve_destroy", "psolve_instance_offset",
           "psolve_total_elements", "psolve_get_status", "psolve_debug_kvec",
           "psolve_error_norms", "psolve_autotune", "psolve_set_profiling", "psolve_pass_times", "psolve_pass_name",
           "psolve_set_operator",
           "psolve_launches_per_solve", "psolve_debug_set_wait", "psolve_debug_tc_dft16",
           "psolve_execute_noalloc", "psolve_status_string",
           "psolve_last_error", "psolve_version")


class PsolveError(RuntimeError):
    def __init__(self, code: int, where: str, message: str):
        self.code = code
        super().__init__(f"{where}: {STATUS.get(code, code)}: {message}")


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load libpsolve.so and declare the C signatures.  Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None and path is None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"{p} is missing: build it with paper_1408_6497_gb300.build.build() "
                               "(needs nvcc); there is no CPU fallback")
        lib = ctypes.CDLL(p)
        vp, i, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_size_t
        pp = ctypes.POINTER(ctypes.c_void_p)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.psolve_plan_create.argtypes = [i, i, i, i, i, pp]
        lib.psolve_plan_create_many.argtypes = [ip, ip, ip, i, i, pp]
        for name in ("psolve_execute", "psolve_adjoint", "psolve_execute_host", "psolve_execute_host_async"):
            getattr(lib, name).argtypes = [vp, vp, vp, vp]
        lib.psolve_destroy.argtypes = [vp]
        lib.psolve_instance_offset.argtypes = [vp, i]
        lib.psolve_instance_offset.restype = sz
        lib.psolve_total_elements.argtypes = [vp]
        lib.psolve_total_elements.restype = sz
        lib.psolve_get_status.argtypes = [vp, vp]
        lib.psolve_debug_kvec.argtypes = [vp, i, ip]
        lib.psolve_error_norms.argtypes = [vp, vp, sz, i, ctypes.POINTER(ctypes.c_double), vp]
        lib.psolve_autotune.argtypes = [vp, vp]
        lib.psolve_set_profiling.argtypes = [vp, i]
        lib.psolve_set_operator.argtypes = [vp, i, ctypes.c_double]
        lib.psolve_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i, ip, ip]
        lib.psolve_pass_name.argtypes = [vp, i]
        lib.psolve_pass_name.restype = ctypes.c_char_p
        lib.psolve_launches_per_solve.argtypes = [vp]
        lib.psolve_launches_per_solve.restype = i
        lib.psolve_execute_noalloc.argtypes = [i, i, i, i, vp, vp, vp]
        lib.psolve_debug_set_wait.argtypes = [vp, ctypes.c_ulonglong, i]
        lib.psolve_debug_tc_dft16.argtypes = [vp, vp, i, i, vp]
        lib.psolve_status_string.argtypes = [i]
        lib.psolve_status_string.restype = ctypes.c_char_p
        lib.psolve_last_error.restype = ctypes.c_char_p
        lib.psolve_version.restype = i
        for name in EXPORTS:
            if name not in ("psolve_instance_offset", "psolve_total_elements", "psolve_status_string",
                            "psolve_last_error", "psolve_version", "psolve_pass_name",
                            "psolve_launches_per_solve"):
                getattr(lib, name).restype = i
        if path is None:
            _lib = lib
        return lib


def check(code: int, where: str) -> None:
    if code != 0:
        msg = load().psolve_last_error().decode(errors="replace")
        raise PsolveError(code, where, msg)
