"""Planted mistakes in the oracle must each fail at least one pin (CPU only).

poisson_oracle.c carries compile-time variants (ORACLE_MUTANT = 1..9) with one
plausible slip each: the 4π² factor dropped, the twiddle sign flipped, the
wavenumber wrap-around forgotten, the x and y axes swapped in the symbol, the
Nyquist mode dropped, the wrong normalisation, a wrong twiddle index, the
finite-difference eigenvalue taken at 2k, the Helmholtz shift replaced.  Each is
built into a temporary library and run through a set of the pins.
"""
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

MUTANTS = {1: "4π² dropped", 2: "twiddle sign", 3: "no wrap-around", 4: "axes swapped",
           5: "Nyquist dropped", 6: "normalisation", 7: "twiddle index",
           8: "finite-difference eigenvalue of 2k", 9: "Helmholtz shift replaced"}


def _pin_suite(mod):
    yield lambda: pins.test_bruteforce_kronecker(mod, (6, 4, 8), False)
    yield lambda: pins.test_bruteforce_kronecker(mod, (4, 6, 6), True)
    yield lambda: pins.test_mode_sum_closed_form_noncubic(mod, (16, 24, 12))
    yield lambda: pins.test_single_modes_every_octant_and_nyquist(mod, (6, 10, 4))
    yield lambda: pins.test_kvec_convention(mod, 8)
    yield lambda: pins.test_parseval_and_hermitian(mod, (12, 6, 16))
    yield lambda: pins.test_fd_operator_solves_the_7_point_stencil(mod, (8, 6, 4))
    yield lambda: pins.test_helmholtz_modes_and_constant(mod, 3.7)


@pytest.mark.parametrize("mutant", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, mutant):
    so = os.path.join(tmp_path, f"liboracle_m{mutant}.so")
    subprocess.run(["gcc", "-O1", "-std=c11", "-shared", "-fPIC", f"-DORACLE_MUTANT={mutant}",
                    oracle._SRC, "-o", so, "-lm"], check=True)
    saved = oracle._lib
    oracle._load()
    try:
        oracle._lib = oracle.open_library(so)
        failures = 0
        for pin in _pin_suite(oracle):
            try:
                pin()
            except AssertionError:
                failures += 1
        assert failures > 0, f"mutant {mutant} ({MUTANTS[mutant]}) passed every pin"
    finally:
        oracle._lib = saved if saved is not None else oracle.open_library(oracle.build())
