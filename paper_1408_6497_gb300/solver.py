"""Python face of the C ABI: plans, solves and the autograd wrapper.

PyTorch supplies device memory and the current stream; each call hands raw
device pointers to libpsolve.so, whose kernels do all of the work (§2.1:
forward FFT, division by the Laplacian symbol, inverse FFT).
"""
from __future__ import annotations

import ctypes
import threading
from typing import Sequence, Tuple

import numpy as np
import torch

from . import _lib

_TORCH_DTYPE = {_lib.F64: torch.float64, _lib.F32: torch.float32, _lib.F32_TC: torch.float32}
_NP_DTYPE = {_lib.F64: np.float64, _lib.F32: np.float32, _lib.F32_TC: np.float32}


def _dtype_code(dtype) -> int:
    if isinstance(dtype, int):
        return dtype
    if dtype in (torch.float64, np.float64, "float64"):
        return _lib.F64
    if dtype in (torch.float32, np.float32, "float32"):
        return _lib.F32
    return _lib.DTYPE_CODES[dtype]


def _stream_handle(stream, device) -> int:
    if stream is None:
        stream = torch.cuda.current_stream(device)
    if isinstance(stream, torch.cuda.Stream):
        return int(stream.cuda_stream)
    return int(stream)


OPERATORS = {"poisson": 0, "helmholtz": 1, "fd": 2}


class Plan:
    """A solve plan for `batch` grids of shape (nx, ny, nz), or for a list of
    unequal shapes (`shapes=[...]`).  Owns the device twiddle tables."""

    def __init__(self, shape: Sequence[int] | None = None, dtype="f32", batch: int = 1,
                 shapes: Sequence[Sequence[int]] | None = None, device=None, operator="poisson",
                 c: float = 0.0):
        self.lib = _lib.load()
        self.code = _dtype_code(dtype)
        self.device = torch.device("cuda", torch.cuda.current_device() if device is None
                                   else torch.device(device).index or 0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            if shapes is not None:
                arr = np.asarray(shapes, dtype=np.int32).reshape(-1, 3)
                cols = [np.ascontiguousarray(arr[:, k]) for k in range(3)]
                ptrs = [c.ctypes.data_as(ctypes.POINTER(ctypes.c_int)) for c in cols]
                rc = self.lib.psolve_plan_create_many(*ptrs, len(arr), self.code, ctypes.byref(h))
                self.shapes = [tuple(int(v) for v in row) for row in arr]
            else:
                nx, ny, nz = (int(v) for v in shape)
                rc = self.lib.psolve_plan_create(nx, ny, nz, self.code, int(batch), ctypes.byref(h))
                self.shapes = [(nx, ny, nz)] * int(batch)
        _lib.check(rc, "psolve_plan_create")
        self.handle = h
        self.batch = len(self.shapes)
        self.total = int(self.lib.psolve_total_elements(h))
        self.torch_dtype = _TORCH_DTYPE[self.code]
        self.np_dtype = _NP_DTYPE[self.code]
        if operator != "poisson":
            self.set_operator(operator, c)

    def set_operator(self, operator="poisson", c: float = 0.0) -> None:
        """The operator later solves invert: "poisson" (−Δu = f), "helmholtz"
        (−Δu + c·u = f, c > 0) or "fd" (the 7-point finite-difference
        Laplacian of the grid)."""
        code = OPERATORS[operator] if isinstance(operator, str) else int(operator)
        with torch.cuda.device(self.device):
            rc = self.lib.psolve_set_operator(self.handle, code, float(c))
        _lib.check(rc, "psolve_set_operator")

    # ----------------------------------------------------------------- utils
    def offset(self, b: int) -> int:
        return int(self.lib.psolve_instance_offset(self.handle, int(b)))

    def view(self, flat: torch.Tensor, b: int) -> torch.Tensor:
        o = self.offset(b)
        nx, ny, nz = self.shapes[b]
        return flat[o:o + nx * ny * nz].view(nx, ny, nz)

    def empty(self) -> torch.Tensor:
        return torch.zeros(self.total, dtype=self.torch_dtype, device=self.device)

    def _check_tensor(self, t: torch.Tensor, name: str) -> None:
        if not t.is_cuda or t.dtype != self.torch_dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {self.torch_dtype} CUDA tensor")
        if t.numel() != self.total:
            raise ValueError(f"{name} has {t.numel()} elements, the plan expects {self.total}")

    # ---------------------------------------------------------------- solves
    def execute(self, f: torch.Tensor, u: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """u = A f on the device (u may be f itself)."""
        self._check_tensor(f, "f")
        if u is None:
            u = torch.empty_like(f)
        self._check_tensor(u, "u")
        rc = self.lib.psolve_execute(self.handle, f.data_ptr(), u.data_ptr(),
                                     _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_execute")
        return u

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """grad_f = A^T g (A is symmetric)."""
        self._check_tensor(g, "g")
        if out is None:
            out = torch.empty_like(g)
        self._check_tensor(out, "grad_f")
        rc = self.lib.psolve_adjoint(self.handle, g.data_ptr(), out.data_ptr(),
                                     _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_adjoint")
        return out

    def execute_host(self, f_host: np.ndarray | torch.Tensor, u_host=None, stream=None):
        """Solve from and into HOST memory (copies included); synchronous."""
        if isinstance(f_host, torch.Tensor):
            if u_host is None:
                u_host = torch.empty_like(f_host)
            fp, up, n = f_host.data_ptr(), u_host.data_ptr(), f_host.numel()
        else:
            f_host = np.ascontiguousarray(f_host, dtype=self.np_dtype)
            if u_host is None:
                u_host = np.empty_like(f_host)
            fp, up, n = f_host.ctypes.data, u_host.ctypes.data, f_host.size
        if n != self.total:
            raise ValueError(f"host array has {n} elements, the plan expects {self.total}")
        with torch.cuda.device(self.device):
            rc = self.lib.psolve_execute_host(self.handle, fp, up, _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_execute_host")
        return u_host

    def execute_host_async(self, f_host: torch.Tensor, u_host: torch.Tensor, stream=None) -> torch.Tensor:
        """Enqueue a host-buffer solve without waiting (pinned tensors go
        straight across the host link); rotate over three or more streams to
        overlap consecutive solves, then synchronise them."""
        if f_host.numel() != self.total or u_host.numel() != self.total:
            raise ValueError(f"host tensors must hold {self.total} elements")
        with torch.cuda.device(self.device):
            rc = self.lib.psolve_execute_host_async(self.handle, f_host.data_ptr(), u_host.data_ptr(),
                                                    _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_execute_host_async")
        return u_host

    def status(self, stream=None) -> None:
        rc = self.lib.psolve_get_status(self.handle, _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_get_status")

    def debug_kvec(self, b: int = 0) -> np.ndarray:
        nx, ny, nz = self.shapes[b]
        out = np.empty((nx, ny, nz // 2 + 1, 3), dtype=np.int32)
        rc = self.lib.psolve_debug_kvec(self.handle, int(b), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
        _lib.check(rc, "psolve_debug_kvec")
        return out

    def autotune(self, stream=None) -> None:
        """Time tile/plan candidates on scratch data and keep the fastest
        (persisted in the per-GPU tuning cache)."""
        with torch.cuda.device(self.device):
            rc = self.lib.psolve_autotune(self.handle, _stream_handle(stream, self.device))
        _lib.check(rc, "psolve_autotune")

    def set_profiling(self, every) -> None:
        """Record per-pass events on every `every`-th solve (True: every
        solve; False or 0: stop)."""
        _lib.check(self.lib.psolve_set_profiling(self.handle, int(every)), "psolve_set_profiling")

    def pass_times(self):
        """{pass name: summed ms} over the solves recorded since profiling began,
        and the number of solves; clears the record."""
        ms = (ctypes.c_double * 16)()
        npass, nsol = ctypes.c_int(), ctypes.c_int()
        rc = self.lib.psolve_pass_times(self.handle, ms, 16, ctypes.byref(npass), ctypes.byref(nsol))
        _lib.check(rc, "psolve_pass_times")
        names = [self.lib.psolve_pass_name(self.handle, i).decode() for i in range(npass.value)]
        return {n: ms[i] for i, n in enumerate(names)}, nsol.value

    @property
    def launches_per_solve(self) -> int:
        return int(self.lib.psolve_launches_per_solve(self.handle))

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.check(self.lib.psolve_destroy(self.handle), "psolve_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def error_norms(a: torch.Tensor, ref: torch.Tensor, stream=None) -> Tuple[float, float]:
    """(rel-L2, rel-ℓ∞) of a against ref, reduced in FP64 on the device."""
    if a.shape != ref.shape or a.dtype != ref.dtype:
        raise ValueError("a and ref must match in shape and dtype")
    out = (ctypes.c_double * 4)()
    code = _dtype_code(a.dtype)
    rc = _lib.load().psolve_error_norms(a.contiguous().data_ptr(), ref.contiguous().data_ptr(),
                                        a.numel(), code, out, _stream_handle(stream, a.device))
    _lib.check(rc, "psolve_error_norms")
    sd, sr, md, mr = out[0], out[1], out[2], out[3]
    return (float(np.sqrt(sd / sr)) if sr > 0 else float(np.sqrt(sd)),
            float(md / mr) if mr > 0 else float(md))


_plan_cache: dict = {}
_plan_lock = threading.Lock()


def get_plan(shape, dtype, batch: int, device) -> Plan:
    key = (tuple(int(v) for v in shape), _dtype_code(dtype), int(batch), str(device))
    with _plan_lock:
        p = _plan_cache.get(key)
        if p is None:
            p = Plan(shape, dtype=dtype, batch=batch, device=device)
            _plan_cache[key] = p
        return p


class PoissonSolve(torch.autograd.Function):
    """u = A f with A = F^{-1} D F; backward gives A^T g = A g (psolve_adjoint)."""

    @staticmethod
    def forward(ctx, f: torch.Tensor, precision: str):
        shape = f.shape[-3:]
        batch = int(np.prod(f.shape[:-3])) if f.dim() > 3 else 1
        plan = get_plan(shape, precision if precision != "auto" else f.dtype, batch, f.device)
        fc = f.contiguous()
        u = plan.execute(fc.view(-1))
        ctx.plan = plan
        return u.view(f.shape)

    @staticmethod
    def backward(ctx, g: torch.Tensor):
        gc = g.contiguous()
        grad = ctx.plan.adjoint(gc.view(-1))
        return grad.view(g.shape), None


def poisson_solve(f: torch.Tensor, precision: str = "auto") -> torch.Tensor:
    """Solve -Δu = f, periodic on [0,1)^3, for f of shape (..., nx, ny, nz)
    on a CUDA device; differentiable in f.  `precision` is "auto" (from
    f.dtype), "f64", "f32" or "f32_tc"."""
    if not f.is_cuda:
        raise ValueError("poisson_solve runs on a CUDA device only")
    return PoissonSolve.apply(f, precision)
