"""GB300-native spectral Poisson solver: -Δu = f, periodic on the unit cube.

`poisson_solve(f)` and `Plan` call libpsolve.so (hand-written sm_103a CUDA
kernels behind the C ABI in include/psolve.h); see solver.py.
"""
from .solver import Plan, PoissonSolve, error_norms, get_plan, poisson_solve  # noqa: F401

__all__ = ["Plan", "PoissonSolve", "error_norms", "get_plan", "poisson_solve"]
