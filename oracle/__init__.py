"""FP64 CPU oracle for the spectral Poisson solve (§1 Eq. 1.1, §2.1, §3).

TEST INFRASTRUCTURE ONLY: imported by tests/, by __graft_entry__.smoke() and by
bench.py's CPU-baseline leg.  The product package never imports it.

`solve(f)` computes the plain definition  u = F^{-1}[ D · F f ],
D(k) = 1/(4π²|k|²), D(0) = 0, in float64 through liboracle.so (C, built from
poisson_oracle.c by `build()`), with either the direct O(n²) DFT per axis or a
plain recursive radix-2/3 FFT.  Everything else here is a thin numpy layer.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "poisson_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (OpenMP if available).  Idempotent."""
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB)
    return _LIB


def open_library(path: str):
    """Load a build of poisson_oracle.c and declare its entry points."""
    lib = ctypes.CDLL(path)
    P = ctypes.POINTER
    lib.oracle_solve.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                 P(ctypes.c_double)]
    lib.oracle_solve.restype = ctypes.c_int
    lib.oracle_solve_op.argtypes = [P(ctypes.c_double), P(ctypes.c_double), ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_double, P(ctypes.c_double)]
    lib.oracle_solve_op.restype = ctypes.c_int
    lib.oracle_op_inverse.argtypes = [ctypes.c_int, ctypes.c_double] + [ctypes.c_int] * 6
    lib.oracle_op_inverse.restype = ctypes.c_double
    lib.oracle_dft3d.argtypes = [P(ctypes.c_double), ctypes.c_int, ctypes.c_int,
                                 ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.oracle_dft3d.restype = None
    lib.oracle_kvec.argtypes = [ctypes.c_int, ctypes.c_int]
    lib.oracle_kvec.restype = ctypes.c_int
    lib.oracle_symbol_inverse.argtypes = [ctypes.c_int] * 6
    lib.oracle_symbol_inverse.restype = ctypes.c_double
    lib.oracle_set_threads.argtypes = [ctypes.c_int]
    lib.oracle_get_threads.restype = ctypes.c_int
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = open_library(build())
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def set_threads(n: int) -> None:
    """Number of OpenMP threads the oracle uses (0 = the runtime default)."""
    _load().oracle_set_threads(int(n))


def threads() -> int:
    return int(_load().oracle_get_threads())


OPS = {"poisson": 0, "helmholtz": 1, "fd": 2}


def solve(f: np.ndarray, direct: bool = False, return_imag: bool = False, op: str = "poisson",
          c: float = 0.0):
    """u = F^{-1}[F[f] / (4π²|k|²)], û(0) = 0, in float64 (§2.1, §3); with
    op="helmholtz" the multiplier is 1/(4π²|k|² + c) (−Δu + c·u = f), with
    op="fd" the inverse eigenvalues of the 7-point finite-difference
    Laplacian."""
    f64 = np.ascontiguousarray(f, dtype=np.float64)
    if f64.ndim != 3:
        raise ValueError("f must be 3D (nx, ny, nz)")
    u = np.empty_like(f64)
    mi = ctypes.c_double(0.0)
    rc = _load().oracle_solve_op(_dptr(f64), _dptr(u), *f64.shape, int(direct), OPS[op], float(c),
                                 ctypes.byref(mi))
    if rc != 0:
        raise MemoryError("oracle_solve: allocation failed")
    return (u, mi.value) if return_imag else u


def dft3d(a: np.ndarray, inverse: bool = False, direct: bool = False) -> np.ndarray:
    """Unscaled 3D DFT, sign -1 forward / +1 inverse, of a complex array."""
    c = np.array(a, dtype=np.complex128, order="C", copy=True)
    if c.ndim != 3:
        raise ValueError("a must be 3D")
    view = c.view(np.float64)
    _load().oracle_dft3d(_dptr(view), *c.shape, 1 if inverse else -1, int(direct))
    return c


def kvec(n: int) -> np.ndarray:
    """Signed integer wavenumbers k(j) of the n indices of one axis."""
    lib = _load()
    return np.array([lib.oracle_kvec(j, n) for j in range(n)], dtype=np.int64)


def symbol_inverse(shape) -> np.ndarray:
    """D(k) = 1/(4π²|k|²), D(0) = 0, on the full (nx, ny, nz) index grid."""
    nx, ny, nz = shape
    kx, ky, kz = kvec(nx), kvec(ny), kvec(nz)
    k2 = (kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2).astype(np.float64)
    with np.errstate(divide="ignore"):
        d = 1.0 / (4.0 * np.pi ** 2 * k2)
    d[0, 0, 0] = 0.0
    return d


def gradient(f: np.ndarray, u_target: np.ndarray) -> np.ndarray:
    """∇_f of ½‖A f − u_t‖² where A is the solve operator.  A is real and
    symmetric (D is real and even in k), so the gradient is A (A f − u_t)."""
    r = solve(f) - np.asarray(u_target, dtype=np.float64)
    return solve(r)


def rel_l2(x: np.ndarray, ref: np.ndarray) -> float:
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.sqrt((ref * ref).sum()))
    return float(np.sqrt(((x - ref) ** 2).sum())) / (den if den > 0 else 1.0)


def rel_linf(x: np.ndarray, ref: np.ndarray) -> float:
    """Relative discrete ℓ∞ error, the paper's accuracy metric (§3)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.abs(ref).max())
    return float(np.abs(x - ref).max()) / (den if den > 0 else 1.0)
