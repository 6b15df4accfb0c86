"""The gradient of loss = ½‖u − u_t‖², u = A f, through the adjoint solve
under torch.autograd, in FP32 and on the tensor-core path, against the FP64
oracle's gradient A(A f − u_t) and against central differences of the loss.

The oracle sees the same rounded f and u_t as the device.  The loss is
exactly quadratic in f, so a central difference has no truncation error at
any step h; h is taken so that h·d is as large as f, which keeps the
rounding of the perturbed FP32 input at the FP32 level relative to the
difference.  The directions lean on the gradient (d = ĝ + ½ r̂, unit ĝ
along the oracle gradient, r̂ a unit random field) so that the directional
derivative is not a small difference of large numbers.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1408_6497_gb300 import poisson_solve
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    oracle.build()


def _gradient_case(shape, prec, fd_tol):
    f32 = wl.sharp_source(shape).f.astype(np.float32)
    ut32 = (wl.smooth_target(shape).f * 1e-3).astype(np.float32)
    f = torch.from_numpy(f32).cuda().requires_grad_(True)
    target = torch.from_numpy(ut32).cuda()
    u = poisson_solve(f, prec)
    loss = 0.5 * ((u - target) ** 2).sum()
    loss.backward()
    g = f.grad.detach()
    g_or = oracle.gradient(f32.astype(np.float64), ut32.astype(np.float64))
    errs = check(g.cpu().numpy(), g_or, prec, f"gradient {shape} {prec}")

    def L(v):
        with torch.no_grad():
            r = poisson_solve(v.float().contiguous(), prec).double() - target.double()
            return 0.5 * float((r * r).sum())

    rng = np.random.default_rng(11)
    gh = g_or / np.linalg.norm(g_or)
    fn = np.linalg.norm(f32.astype(np.float64))
    worst = 0.0
    for _ in range(3):
        r = rng.standard_normal(shape)
        d = gh + 0.5 * r / np.linalg.norm(r)
        h = fn / np.linalg.norm(d)
        dd = torch.from_numpy(d).cuda()
        fd = (L(f.detach().double() + h * dd) - L(f.detach().double() - h * dd)) / (2 * h)
        an = float((g.double() * dd).sum())
        worst = max(worst, abs(fd - an) / abs(an))
    print(f"gradient {shape} {prec}: (rel-L2, rel-linf) vs oracle {errs}, worst central-difference "
          f"relative gap {worst:.2e}")
    assert worst <= fd_tol
    return g


def test_gradient_64_fp32_vs_oracle_and_fd():
    _gradient_case((64, 64, 64), "f32", 1e-4)


def test_gradient_tensor_cores_vs_oracle_and_fd():
    """256 × 256 × 64: the y and x lines (256 points) run their radix-16
    stages on the tensor cores, in the forward solve and in the adjoint."""
    from paper_1408_6497_gb300.solver import get_plan
    shape = (256, 256, 64)
    _gradient_case(shape, "f32_tc", 1e-4)
    plan = get_plan(shape, "f32_tc", 1, torch.device("cuda", torch.cuda.current_device()))
    names = [plan.lib.psolve_pass_name(plan.handle, i).decode() for i in range(5)]
    assert names == ["zfwd", "yfwd_tc", "xdiv_tc", "yinv_tc", "zinv"]
