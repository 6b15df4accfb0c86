"""Relative ℓ∞ error of the FP64 oracle's solve of the sharp-layer case (§3,
test case 2) at the grids of the paper's FFT figures (Tables 8 and 9,
tests/golden/paper_table8_9_fft.txt), for a given sphere radius R:

    python tests/golden/sphere_radius_table.py [--radius 0.1] [--large]

--large adds α = 40 at 512³, 768³ and 1024³ (minutes of oracle time and
about 40 GB of host memory at 1024³).  Prints one JSON line per grid.
"""
import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1408_6497_gb300 import workloads as wl  # noqa: E402

SLAB = 32


def rel_linf(n, alpha, R):
    """Error of the oracle's u against u minus its mean, the source and the
    exact u evaluated slab by slab along x so that large grids fit."""
    f = np.empty((n, n, n))
    usum = 0.0
    for x0 in range(0, n, SLAB):
        fs, us = wl.sphere_layer((n, n, n), alpha, R=R, rows=(x0, min(n, x0 + SLAB)))
        f[x0:x0 + SLAB] = fs
        usum += us.sum()
    mean = usum / n ** 3
    uN = oracle.solve(f)
    del f
    emax = umax = 0.0
    for x0 in range(0, n, SLAB):
        _, us = wl.sphere_layer((n, n, n), alpha, R=R, rows=(x0, min(n, x0 + SLAB)))
        ue = us - mean
        emax = max(emax, float(np.abs(uN[x0:x0 + SLAB] - ue).max()))
        umax = max(umax, float(np.abs(ue).max()))
    return emax / umax


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--radius", type=float, default=0.1)
    ap.add_argument("--large", action="store_true")
    args = ap.parse_args()
    oracle.build()
    cases = [(40.0, 384), (10.0, 128), (10.0, 192), (10.0, 256)]
    if args.large:
        cases += [(40.0, 512), (40.0, 768), (40.0, 1024)]
    for alpha, n in cases:
        t0 = time.perf_counter()
        e = rel_linf(n, alpha, args.radius)
        print(json.dumps({"alpha": alpha, "n": n, "R": args.radius, "rel_linf": e,
                          "oracle_threads": oracle.threads(), "seconds": round(time.perf_counter() - t0, 1)}),
              flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
