"""The C ABI library builds, loads and exports every declared symbol; the
host-side argument checks answer without a GPU (CPU only)."""
import ctypes
import os
import re
import subprocess
import sys

import pytest
import torch

from paper_1408_6497_gb300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "psolve.h")


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _lib.load()


def declared_symbols():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"\b(psolve_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(_lib.EXPORTS)


def test_version_and_status_strings(lib):
    assert lib.psolve_version() == 100
    assert lib.psolve_status_string(0) == b"ok"
    assert lib.psolve_status_string(2) == b"unsupported size"


@pytest.mark.parametrize("dims", [(5, 8, 8), (8, 7, 8), (8, 8, 10), (2, 8, 8), (4096, 4, 4),
                                  (8, 8, 14), (9, 8, 8), (0, 8, 8), (-4, 8, 8)])
def test_unsupported_sizes_rejected_before_any_cuda_call(lib, dims):
    h = ctypes.c_void_p(123)
    rc = lib.psolve_plan_create(*dims, _lib.F32, 1, ctypes.byref(h))
    assert rc == 2
    assert h.value is None
    assert b"2^a 3^b" in lib.psolve_last_error()


def test_fp64_x_lines_of_1458_points_rejected(lib):
    # the x pass's tile of two 1458-point FP64 lines needs 486 threads; the
    # plan says so before any CUDA call (FP32 takes the same grid)
    h = ctypes.c_void_p()
    assert lib.psolve_plan_create(1458, 8, 8, _lib.F64, 1, ctypes.byref(h)) == 2
    assert b"1458" in lib.psolve_last_error()
    ok = (ctypes.c_int * 2)(1458, 8)
    eight = (ctypes.c_int * 2)(8, 8)
    assert lib.psolve_plan_create_many(ok, eight, eight, 2, _lib.F64, ctypes.byref(h)) == 2


def test_bad_arguments_rejected(lib):
    h = ctypes.c_void_p()
    assert lib.psolve_plan_create(8, 8, 8, _lib.F32, 0, ctypes.byref(h)) == 1
    assert lib.psolve_plan_create(8, 8, 8, 9, 1, ctypes.byref(h)) == 1
    assert lib.psolve_plan_create(8, 8, 8, _lib.F32, 1, None) == 1
    assert lib.psolve_execute(None, None, None, None) == 1
    assert lib.psolve_adjoint(None, None, None, None) == 1
    assert lib.psolve_destroy(None) == 1
    assert lib.psolve_instance_offset(None, 0) == ctypes.c_size_t(-1).value
    assert lib.psolve_total_elements(None) == 0
    arr = (ctypes.c_int * 2)(8, 7)
    ok = (ctypes.c_int * 2)(8, 8)
    assert lib.psolve_plan_create_many(ok, arr, ok, 2, _lib.F32, ctypes.byref(h)) == 2
    assert b"instance 1" in lib.psolve_last_error()


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-device path")
def test_valid_plan_without_device_fails_loudly(lib):
    h = ctypes.c_void_p()
    rc = lib.psolve_plan_create(8, 8, 8, _lib.F32, 1, ctypes.byref(h))
    assert rc == 4  # PSOLVE_ERR_CUDA, not a silent CPU path
    assert h.value is None


def test_binding_raises_when_library_missing(tmp_path):
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        _lib.load(str(tmp_path / "libpsolve.so"))


def _noalloc_refusals():
    """Every case below is refused before any CUDA call; the made-up
    pointers are never dereferenced.  The call leaves psolve_last_error()
    alone (it sets no message, so it allocates nothing on the host either)."""
    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.psolve_plan_create(10, 8, 8, _lib.F32, 1, ctypes.byref(h)) == 2
    before = lib.psolve_last_error()
    assert before
    a = ctypes.c_void_p(1 << 20)
    b = ctypes.c_void_p((1 << 20) + (1 << 16))
    F32, F64 = _lib.F32, _lib.F64
    assert lib.psolve_execute_noalloc(8, 8, 8, 9, a, b, None) == 1            # unknown dtype
    assert lib.psolve_execute_noalloc(8, 8, 8, _lib.F32_TC, a, b, None) == 1  # TC needs a plan
    assert lib.psolve_execute_noalloc(10, 8, 8, F32, a, b, None) == 2         # 10 = 2·5
    assert lib.psolve_execute_noalloc(8, 8, 4096, F32, a, b, None) == 2       # above 2048
    # FP64 tables for nx + ny + nz = 4100 points: 65600 bytes > 64 KiB
    assert lib.psolve_execute_noalloc(2048, 2048, 4, F64, a, b, None) == 2
    assert lib.psolve_execute_noalloc(8, 8, 8, F32, None, b, None) == 1       # null f
    assert lib.psolve_execute_noalloc(8, 8, 8, F32, a, None, None) == 1       # null u
    odd = ctypes.c_void_p((1 << 20) + 8)
    assert lib.psolve_execute_noalloc(8, 8, 8, F32, odd, b, None) == 1        # not 16-B aligned
    # u starts 16 bytes into f's 2 KiB (8³ FP32): partial overlap
    inside = ctypes.c_void_p((1 << 20) + 16)
    assert lib.psolve_execute_noalloc(8, 8, 8, F32, a, inside, None) == 1
    assert lib.psolve_last_error() == before


def test_noalloc_argument_checks_on_the_host(lib):
    # Run with no device visible, so that even a host check that stopped
    # working could only end in a CUDA error, never in a launch on made-up
    # addresses.
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    code = "import tests.test_abi as t; t._noalloc_refusals(); print('refusals ok')"
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "refusals ok" in r.stdout


def test_every_plan_entry_point_rejects_a_null_plan(lib):
    # answered on the host before any CUDA call (no device here)
    for name in ("psolve_execute", "psolve_adjoint", "psolve_execute_host", "psolve_execute_host_async"):
        assert getattr(lib, name)(None, None, None, None) == 1, name
    assert lib.psolve_set_operator(None, 0, 0.0) == 1
    assert lib.psolve_get_status(None, None) == 1
    assert lib.psolve_debug_kvec(None, 0, None) == 1
    assert lib.psolve_autotune(None, None) == 1
    assert lib.psolve_set_profiling(None, 1) == 1
    assert lib.psolve_pass_times(None, None, 0, None, None) == 1
    assert lib.psolve_debug_set_wait(None, 0, 0) == 1
    assert lib.psolve_pass_name(None, 0) is None
    assert lib.psolve_launches_per_solve(None) == 0
    assert b"invalid or destroyed plan" in lib.psolve_last_error()
    # pointer checks of the plan-free helpers
    assert lib.psolve_error_norms(None, None, 0, _lib.F32, None, None) == 1
    assert lib.psolve_debug_tc_dft16(None, None, 0, 0, None) == 1
