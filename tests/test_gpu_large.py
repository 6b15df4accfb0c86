"""Full-size checks at 1024^3 (FP32 and the tensor-core path): a plane-wave
sum whose exact solution is known in closed form is solved on the device and
compared with the closed form at EVERY grid point.

The input is built on the device from per-axis factors (plane waves factor
over the axes) because a 1024^3 FP64 array does not fit comfortably in host
memory; the exact solution is evaluated on the device in FP64 the same way,
one slab of x-planes at a time, and the error norms are accumulated in FP64.
The per-axis factors come from numpy in FP64.
"""
import numpy as np
import pytest
import torch

from paper_1408_6497_gb300 import Plan

from .tolerances import TOL, TOL_INF

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()


def _factors(k, phi, n):
    """Per mode: (sin, cos) of 2πk_x x + φ, of 2πk_y y and of 2πk_z z on the
    grid, FP64 on the device."""
    x = np.arange(n) / n
    out = []
    for (kx, ky, kz), pm in zip(k, phi):
        A, B, C = 2 * np.pi * kx * x + pm, 2 * np.pi * ky * x, 2 * np.pi * kz * x
        out.append([torch.from_numpy(v).cuda() for v in (np.sin(A), np.cos(A), np.sin(B), np.cos(B),
                                                         np.sin(C), np.cos(C))])
    return out


def _mode_sum(fac, coef, x0, x1):
    """Σ_m coef_m sin(2π k_m·x + φ_m) over x-planes [x0, x1), FP64, by
    sin(A+B+C) = sA cB cC + cA sB cC + cA cB sC - sA sB sC."""
    out = None
    for (sa, ca, sb, cb, sc, cc), c in zip(fac, coef):
        sa, ca = sa[x0:x1], ca[x0:x1]
        t = sa[:, None, None] * cb[None, :, None] * cc[None, None, :]
        t += ca[:, None, None] * sb[None, :, None] * cc[None, None, :]
        t += ca[:, None, None] * cb[None, :, None] * sc[None, None, :]
        t -= sa[:, None, None] * sb[None, :, None] * sc[None, None, :]
        t *= c
        out = t if out is None else out.add_(t)
    return out


@pytest.mark.parametrize("prec", ["f32", "f32_tc"])
def test_1024_cubed_closed_form_full_grid(prec):
    n, slab = 1024, 64
    rng = np.random.default_rng(1024)
    k = rng.integers(-500, 501, size=(8, 3))
    k[np.all(k == 0, axis=1)] = 1
    a, phi = rng.standard_normal(8), rng.uniform(0, 2 * np.pi, 8)
    fac = _factors(k, phi, n)
    f = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    for x0 in range(0, n, slab):
        f[x0:x0 + slab] = _mode_sum(fac, a, x0, x0 + slab).float()
    plan = Plan((n, n, n), dtype=prec)
    u = plan.execute(f.view(-1), f.view(-1)).view(n, n, n)  # in place: 4 GiB
    plan.status()
    # exact u = Σ a_m / (4π²|k_m|²) sin(2π k_m·x + φ_m): |k_i| ≤ 500 < 512, so
    # the grid resolves every mode and the discrete solution equals it
    coef = [am / (4 * np.pi ** 2 * float(km @ km)) for km, am in zip(k, a)]
    se = sr = me = mr = 0.0
    for x0 in range(0, n, slab):
        ex = _mode_sum(fac, coef, x0, x0 + slab)
        d = u[x0:x0 + slab].double() - ex
        se += float((d * d).sum())
        sr += float((ex * ex).sum())
        me = max(me, float(d.abs().max()))
        mr = max(mr, float(ex.abs().max()))
        del ex, d
    l2, linf = (se / sr) ** 0.5, me / mr
    print(f"1024^3 {prec}: full-grid rel-L2 {l2:.2e}, rel-linf {linf:.2e}")
    assert l2 <= TOL[prec]
    assert linf <= TOL_INF[prec]
    assert abs(float(u.double().mean())) <= 1e-6 * float(u.abs().max())
