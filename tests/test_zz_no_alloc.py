"""psolve_execute_noalloc, the allocation-free solve, through the C ABI.

Callers that cannot allocate device memory (code inside an allocator or
memory-pool callback, frameworks that forbid allocation during a step, hosts
that reserve all device memory up front) use this entry point: it keeps its
twiddle tables in a fixed 64 KiB array inside the library instead of a plan.
Its result must match psolve_execute's, call after call, even though every
call reuses the same shared array, and the FP64 oracle's within the parity
tolerances.  This file is collected last on purpose.
"""

import numpy as np
import pytest
import torch

import oracle
from paper_1408_6497_gb300 import Plan, _lib
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import check

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 5e-6}
NP = {"f64": np.float64, "f32": np.float32}
CODE = {"f64": _lib.F64, "f32": _lib.F32}


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    return _lib.load()


def rel_l2(a, b):
    a = a.double()
    b = b.double()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def noalloc_solve(lib, prec, shape, f):
    u = torch.empty_like(f)
    stream = torch.cuda.current_stream().cuda_stream
    rc = lib.psolve_execute_noalloc(*shape, CODE[prec], f.data_ptr(), u.data_ptr(), stream)
    assert rc == 0, _lib.STATUS.get(rc, rc)
    torch.cuda.synchronize()
    return u


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_noalloc_matches_planned_solve_on_consecutive_calls(lib, prec):
    # Two different grids, then the first again: the shared table array is
    # rewritten by each call, so no call may see the previous call's tables.
    shapes = [(48, 32, 96), (24, 64, 18), (48, 32, 96)]
    for i, shape in enumerate(shapes):
        f = torch.from_numpy(wl.random_field(shape, seed=900 + i).astype(NP[prec]).ravel()).cuda()
        ref = Plan(shape, dtype=prec).execute(f)
        u = noalloc_solve(lib, prec, shape, f)
        err = rel_l2(u, ref)
        assert err <= TOL[prec], (shape, prec, err)
        check(u.cpu().numpy().reshape(shape), oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape)),
              prec, shape)


def test_noalloc_in_place_and_twice_in_a_row(lib):
    shape = (32, 32, 32)
    f = torch.from_numpy(wl.mode_sum(shape).f.astype(np.float32).ravel()).cuda()
    ref = Plan(shape, dtype="f32").execute(f)
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        g = f.clone()
        rc = lib.psolve_execute_noalloc(*shape, _lib.F32, g.data_ptr(), g.data_ptr(), stream)
        assert rc == 0
        torch.cuda.synchronize()
        assert rel_l2(g, ref) <= TOL["f32"]


def test_noalloc_rejects_grids_beyond_the_table_array(lib):
    # FP64 tables for nx + ny + nz = 4100 need 65600 bytes > 64 KiB: refused
    # on the host before anything is enqueued.  Size and dtype checks come
    # before the pointer checks, so null arrays are passed: a size check that
    # stopped working would end in the null-pointer refusal, not a launch.
    assert lib.psolve_execute_noalloc(2048, 2048, 4, _lib.F64, None, None, None) == 2
    # sizes outside the solver's range (10 = 2·5) and the tensor-core dtype
    # (which needs a plan) are refused the same way
    assert lib.psolve_execute_noalloc(10, 8, 8, _lib.F32, None, None, None) == 2
    assert lib.psolve_execute_noalloc(8, 8, 8, _lib.F32_TC, None, None, None) == 1


@pytest.mark.parametrize("prec,shape", [("f32", (2048, 2048, 4)), ("f64", (2048, 1024, 8))])
def test_noalloc_grids_near_the_table_limit(lib, prec, shape):
    # FP32 (2048, 2048, 4): 4100 complex twiddles = 32.8 KB of the 64 KiB
    # array (every FP32 grid fits); FP64 (2048, 1024, 8): 3080 complex
    # twiddles = 49.3 KB, within the FP64 limit nx + ny + nz <= 4096
    f = torch.from_numpy(wl.random_field(shape, seed=77).astype(NP[prec]).ravel()).cuda()
    ref = Plan(shape, dtype=prec).execute(f)
    for _ in range(2):
        u = noalloc_solve(lib, prec, shape, f)
        assert rel_l2(u, ref) <= TOL[prec]
    check(u.cpu().numpy().reshape(shape), oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape)),
          prec, shape)
