"""Other operators on the same passes (Helmholtz −Δu + c·u = f and the
7-point finite-difference Laplacian) against the FP64 oracle, through the
C ABI: every x-pass variant (TMA FP32, per-tile FP32/FP64, tensor cores, the
x-split layout, the batched launch)."""
import numpy as np
import pytest
import torch

import oracle
from paper_1408_6497_gb300 import Plan
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import check

pytestmark = pytest.mark.gpu

OPS = [("helmholtz", 3.7), ("fd", 0.0), ("helmholtz", 250.0)]


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    oracle.build()


def _check(shape, prec, op, c, f64=None, seed=0):
    if f64 is None:
        f64 = wl.random_field(shape, seed=seed + sum(shape))
    np_t = np.float64 if prec == "f64" else np.float32
    plan = Plan(shape, dtype=prec, operator=op, c=c)
    f = torch.from_numpy(f64.astype(np_t).ravel()).cuda()
    u = plan.execute(f)
    plan.status()
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape), op=op, c=c)
    check(u.cpu().numpy().reshape(shape), ref, prec, (shape, prec, op, c))
    return plan, f, u


@pytest.mark.parametrize("op,c", OPS)
@pytest.mark.parametrize("shape,prec", [((512, 256, 32), "f32"), ((256, 512, 64), "f32"),
                                        ((48, 16, 256), "f32"), ((96, 24, 12), "f32"),
                                        ((24, 16, 12), "f64"), ((12, 18, 8), "f64")])
def test_operator_parity(shape, prec, op, c):
    _check(shape, prec, op, c)


@pytest.mark.parametrize("shape", [(16, 54, 2048), (1536, 16, 54), (8, 12, 1728)])
def test_fd_operator_fp64_fine_lines(shape):
    # lowest modes of 1728-2048-point lines: the stencil eigenvalues there
    # are small differences, evaluated without cancellation on both sides
    _check(shape, "f64", "fd", 0.0)


@pytest.mark.parametrize("op,c", OPS[:2])
def test_operator_tensor_cores(op, c):
    _check((512, 512, 32), "f32_tc", op, c)


@pytest.mark.parametrize("op,c", OPS[:2])
def test_operator_xsplit_layout(op, c, monkeypatch):
    monkeypatch.setenv("PSOLVE_XSPLIT", "4")
    _check((256, 256, 512), "f32", op, c)


@pytest.mark.parametrize("op,c", OPS[:2])
def test_operator_batched(op, c):
    shapes = [(24, 32, 48), (64, 24, 96), (32, 32, 32), (48, 128, 24)]
    plan = Plan(dtype="f32", shapes=shapes, operator=op, c=c)
    f = plan.empty()
    fs = [wl.random_field(s, seed=30 + i) for i, s in enumerate(shapes)]
    for b, fb in enumerate(fs):
        plan.view(f, b).copy_(torch.from_numpy(fb.astype(np.float32)))
    u = plan.execute(f)
    plan.status()
    for b, s in enumerate(shapes):
        ref = oracle.solve(plan.view(f, b).cpu().numpy().astype(np.float64), op=op, c=c)
        check(plan.view(u, b).cpu().numpy(), ref, "f32")


def test_switching_operators_and_adjoint():
    shape = (64, 48, 32)
    plan, f, u_h = _check(shape, "f32", "helmholtz", 5.0)
    g = plan.adjoint(f)
    assert torch.allclose(g, u_h, rtol=0, atol=0)  # self-adjoint, same kernels
    plan.set_operator("poisson")
    u_p = plan.execute(f)
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape))
    check(u_p.cpu().numpy().reshape(shape), ref, "f32")
    plan.set_operator("fd")
    u_fd = plan.execute(f)
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape), op="fd")
    check(u_fd.cpu().numpy().reshape(shape), ref, "f32")


@pytest.mark.parametrize("op,c", [(5, 0.0), ("helmholtz", 0.0), ("helmholtz", -1.0),
                                  ("helmholtz", float("nan"))])
def test_operator_argument_errors(op, c):
    plan = Plan((8, 8, 8), dtype="f32")
    with pytest.raises(Exception):
        plan.set_operator(op, c)


def test_sphere_layer_case_on_gpu_matches_oracle():
    """The sharp-layer case of the resolution study, FP64 on the GPU, has the
    oracle's error at the same grid."""
    from paper_1408_6497_gb300 import study
    for n in (32, 64):
        r = study.solve_case(n, 10.0, "f64")
        f, u = wl.sphere_layer((n, n, n), 10.0)
        ue = u - u.mean()
        e_or = np.abs(oracle.solve(f) - ue).max() / np.abs(ue).max()
        assert abs(r["rel_linf"] - e_or) <= 1e-9 * max(e_or, 1.0), (n, r, e_or)
