"""Parity tolerances of the CUDA path against the FP64 oracle, and the check
every parity test applies.

Relative L2 (the stated bounds): FP64 1e-12, FP32 5e-6, tensor-core path
1e-5.  Relative ℓ∞ (the paper's own accuracy metric, §3; Table 7's caption
defines it at the grid points): twice the L2 bound for FP32 and the tensor
cores, the L2 bound itself for FP64.  Why twice: the rounding error of a
solve is spread over all wavenumbers, so its largest point is a few times
its RMS value (about sqrt(2 ln N) <= 6.5 for N up to 1024³), and the
solution, dominated by its lowest modes after the division by |k|², also
peaks at a few times its RMS value; rel-ℓ∞ stays within a small factor of
rel-L2 (measured 1.6 to 3.0 on the workloads here, at errors 10 to 30 times
below the L2 bounds), while an error confined to one tile, which an L2 norm
over a large grid dilutes, still shows in full.
"""
import numpy as np

import oracle

TOL = {"f64": 1e-12, "f32": 5e-6, "f32_tc": 1e-5}
TOL_INF = {"f64": 1e-12, "f32": 1e-5, "f32_tc": 2e-5}


def check(u, ref, prec, what=""):
    """Assert rel-L2 and rel-ℓ∞ of u against ref within the bounds of
    `prec`; returns (rel_l2, rel_linf)."""
    u = np.asarray(u, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    l2, linf = oracle.rel_l2(u, ref), oracle.rel_linf(u, ref)
    assert l2 <= TOL[prec], (what, prec, "rel-L2", l2)
    assert linf <= TOL_INF[prec], (what, prec, "rel-linf", linf)
    return l2, linf
