"""The sharp-layer case (§3 test case 2): the closed-form source against the
FP64 oracle, and the resolution trend the paper states (CPU only)."""
import numpy as np
import pytest

from paper_1408_6497_gb300 import workloads as wl


def _err(oracle_mod, n, alpha):
    f, u = wl.sphere_layer((n, n, n), alpha)
    uN = oracle_mod.solve(f)
    ue = u - u.mean()  # the periodic solve fixes u up to its mean
    return np.abs(uN - ue).max() / np.abs(ue).max()


def test_closed_form_source_is_minus_laplacian(oracle_mod):
    # a well-resolved layer: the spectral solve of the closed-form f returns u
    # (spectral convergence: 7e-6 at 64³, 4e-11 at 128³)
    assert _err(oracle_mod, 128, 10.0) < 1e-9


@pytest.mark.parametrize("alpha", [10.0, 20.0])
def test_error_falls_with_resolution(oracle_mod, alpha):
    e = [_err(oracle_mod, n, alpha) for n in (16, 32, 64)]
    assert e[0] > e[1] > e[2]


def test_doubling_alpha_needs_twice_the_points_per_axis(oracle_mod):
    # the same accuracy at (n, α) and (2n, 2α): the spectrum scales with α
    e1, e2 = _err(oracle_mod, 32, 10.0), _err(oracle_mod, 64, 20.0)
    assert 0.05 < e2 / e1 < 20.0
    assert _err(oracle_mod, 32, 20.0) > 10 * e2  # not enough points for 2α
