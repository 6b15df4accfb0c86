"""Resolution study on the paper's sharp-layer case (§3, test case 2; Tables
8 and 9): u = exp(-(r/R)^α) with f = -Δu in closed form, solved on grids of
growing n until the relative ℓ∞ error (the paper's metric) reaches a target.
The paper's claim to reproduce: each doubling of α doubles the points per
axis the FFT solve needs (eight times the unknowns).

    python -m paper_1408_6497_gb300.study [--alphas 10 20 40] [--target 4e-7] [--radius 0.1]

prints one JSON line per (α, n) and a summary line per α.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np
import torch

from . import workloads as wl
from .solver import Plan

GRIDS = (32, 48, 64, 96, 128, 192, 256, 384, 512, 768, 1024)
SLAB = 32  # x-planes of the closed forms evaluated at a time on the host


def source(n: int, alpha: float, R: float = 0.1, dtype=np.float64):
    """f on the n³ grid, built slab by slab (no full-size temporaries), and
    the mean of the exact u."""
    f = np.empty((n, n, n), dtype=dtype)
    usum = 0.0
    for x0 in range(0, n, SLAB):
        fs, us = wl.sphere_layer((n, n, n), alpha, R=R, rows=(x0, min(n, x0 + SLAB)))
        f[x0:x0 + SLAB] = fs
        usum += float(us.sum())
    return f, usum / n ** 3


def rel_linf(uN: np.ndarray, n: int, alpha: float, R: float, umean: float) -> float:
    """Relative ℓ∞ error of uN against u minus its mean (the periodic solve
    fixes u up to a constant), slab by slab."""
    emax = umax = 0.0
    for x0 in range(0, n, SLAB):
        _, us = wl.sphere_layer((n, n, n), alpha, R=R, rows=(x0, min(n, x0 + SLAB)))
        ue = us - umean
        emax = max(emax, float(np.abs(uN[x0:x0 + SLAB].astype(np.float64) - ue).max()))
        umax = max(umax, float(np.abs(ue).max()))
    return emax / umax


def solve_case(n: int, alpha: float, dtype: str = "f64", R: float = 0.1) -> dict:
    np_t = np.float64 if dtype == "f64" else np.float32
    f, umean = source(n, alpha, R, np_t)
    plan = Plan((n, n, n), dtype=dtype)
    ft = torch.from_numpy(f.reshape(-1)).cuda()
    del f
    uN = plan.execute(ft)  # first solve: plan set-up paid
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uN = plan.execute(ft, uN)
    torch.cuda.synchronize()
    ms = (time.perf_counter() - t0) * 1e3
    plan.status()
    del ft
    err = rel_linf(uN.cpu().numpy().reshape(n, n, n), n, alpha, R, umean)
    return {"alpha": alpha, "R": R, "n": n, "unknowns": n ** 3, "dtype": dtype, "rel_linf": err, "solve_ms": ms}


def resolution(alphas=(10.0, 20.0, 40.0), target: float = 4e-7, dtype: str = "f64", grids=GRIDS,
               R: float = 0.1):
    """For each α, solve on growing grids until rel ℓ∞ <= target; returns
    (rows, {α: smallest n reaching the target or None})."""
    rows, need = [], {}
    for alpha in alphas:
        need[alpha] = None
        for n in grids:
            r = solve_case(n, alpha, dtype, R)
            rows.append(r)
            print(json.dumps(r), flush=True)
            if r["rel_linf"] <= target:
                need[alpha] = n
                break
    return rows, need


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--alphas", type=float, nargs="+", default=[10.0, 20.0, 40.0])
    ap.add_argument("--target", type=float, default=4e-7)
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--radius", type=float, default=0.1,
                    help="sphere radius R (not stated in the paper; 0.1 gives its Tables 8 and 9)")
    args = ap.parse_args(argv)
    _, need = resolution(args.alphas, args.target, args.dtype, R=args.radius)
    for alpha, n in need.items():
        print(json.dumps({"alpha": alpha, "R": args.radius, "target_rel_linf": args.target,
                          "points_per_axis_needed": n, "unknowns": None if n is None else n ** 3}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
