"""Seeded synthetic right-hand sides for the periodic Poisson problem -Δu = f.

The model problem (§1, Eq. 1.1) asks for u given a smooth periodic f on the unit
cube; the paper's own right-hand sides are closed forms (§3: test case 1, an
oscillatory product of sines; test case 2, a sharp spherical layer).  This module
only *draws* inputs: sums of Fourier modes and periodised Gaussians on the grid
x_j = j/n, j = 0..n-1, per axis.  It holds none of the solver's arithmetic (no
transform, no spectral multiplier) so that the GPU path and the FP64 oracle can
both consume the same inputs without sharing any of the method.

Every generator is deterministic in its seed (numpy's PCG64 via default_rng) and
returns float64; callers cast to the dtype under test.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Sequence, Tuple

import numpy as np

SEED_BASE = 20140800  # seed = SEED_BASE + workload index (+ instance for batches)

# Per-axis sizes of the uneven batch (radix-2/3, non-cubic instances).
BATCH_AXIS_CHOICES = (24, 32, 48, 64, 96, 128, 192, 256)


def grid_axis(n: int) -> np.ndarray:
    """Sample points x_j = j/n on the periodic unit interval [0, 1)."""
    return np.arange(n, dtype=np.float64) / n


@dataclass
class ModeSet:
    """A finite sum of plane waves  sum_m a_m sin(2π k_m·x + φ_m)."""
    k: np.ndarray      # (m, 3) integer wave vectors
    a: np.ndarray      # (m,) amplitudes
    phi: np.ndarray    # (m,) phases


@dataclass
class GaussianSet:
    """A sum of Gaussians  sum_g a_g exp(-|x - c_g|^2 / (2 σ_g^2)), periodised."""
    c: np.ndarray      # (g, 3) centres in [0,1)^3
    sigma: np.ndarray  # (g,) widths
    a: np.ndarray      # (g,) amplitudes


@dataclass
class Workload:
    name: str
    shape: Tuple[int, int, int]
    f: np.ndarray                     # float64, C-order (nx, ny, nz); z contiguous
    modes: ModeSet | None = None
    gaussians: GaussianSet | None = None
    mean_subtracted: bool = False
    extra: dict = field(default_factory=dict)


def draw_modes(rng: np.random.Generator, m: int, kmax: int,
               max_norm: float | None = None) -> ModeSet:
    """m wave vectors uniform on {-kmax..kmax}^3 without k = 0 (and, if given,
    with |k| <= max_norm); a ~ N(0,1); φ ~ U[0, 2π)."""
    ks = []
    while len(ks) < m:
        k = rng.integers(-kmax, kmax + 1, size=3)
        if not k.any():
            continue
        if max_norm is not None and float(np.sqrt((k * k).sum())) > max_norm:
            continue
        ks.append(k)
    k = np.array(ks, dtype=np.int64)
    a = rng.standard_normal(m)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=m)
    return ModeSet(k=k, a=a, phi=phi)


def eval_modes(ms: ModeSet, shape: Sequence[int]) -> np.ndarray:
    """Samples of sum_m a_m sin(2π k_m·x + φ_m) on the grid.

    Each plane wave factorises over the axes, e^{i(2π k·x + φ)} =
    e^{iφ} e^{2πi kx x} e^{2πi ky y} e^{2πi kz z}, so it is built as an outer
    product of three 1D vectors (cheap at 512^3) and the imaginary part taken.
    """
    nx, ny, nz = shape
    f = np.zeros(shape, dtype=np.float64)
    ax = [grid_axis(n) for n in shape]
    for (kx, ky, kz), a, phi in zip(ms.k, ms.a, ms.phi):
        ex = np.exp(2j * np.pi * kx * ax[0]) * (a * np.exp(1j * phi))
        ey = np.exp(2j * np.pi * ky * ax[1])
        ez = np.exp(2j * np.pi * kz * ax[2])
        f += np.imag(ex[:, None, None] * (ey[:, None] * ez[None, :])[None, :, :])
    return f


def periodic_gaussian_1d(x: np.ndarray, c: float, sigma: float) -> np.ndarray:
    """sum over images s in {-1,0,1} of exp(-(x - c + s)^2 / (2 σ^2)).

    For σ <= 0.1 the next images (|shift| >= 2 - 1 = 1 away from any sample)
    contribute below exp(-50), far under double-precision rounding."""
    out = np.zeros_like(x)
    for s in (-1.0, 0.0, 1.0):
        d = x - c + s
        out += np.exp(-(d * d) / (2.0 * sigma * sigma))
    return out


def eval_gaussians(gs: GaussianSet, shape: Sequence[int]) -> np.ndarray:
    """Samples of the periodised Gaussian sum.  The 27-image sum of a 3D
    Gaussian is the product of three 1D image sums, so each term is an outer
    product of three axis vectors."""
    ax = [grid_axis(n) for n in shape]
    f = np.zeros(tuple(shape), dtype=np.float64)
    for c, s, a in zip(gs.c, gs.sigma, gs.a):
        gx = periodic_gaussian_1d(ax[0], c[0], s) * a
        gy = periodic_gaussian_1d(ax[1], c[1], s)
        gz = periodic_gaussian_1d(ax[2], c[2], s)
        f += gx[:, None, None] * (gy[:, None] * gz[None, :])[None, :, :]
    return f


def draw_gaussians(rng: np.random.Generator, g: int, sigma) -> GaussianSet:
    """g centres ~ U[0,1)^3, amplitudes ~ N(0,1); sigma is a float or a
    (lo, hi) pair drawn uniformly per Gaussian."""
    c = rng.uniform(0.0, 1.0, size=(g, 3))
    a = rng.standard_normal(g)
    if isinstance(sigma, tuple):
        s = rng.uniform(sigma[0], sigma[1], size=g)
    else:
        s = np.full(g, float(sigma))
    return GaussianSet(c=c, sigma=s, a=a)


# --------------------------------------------------------------------------
# The five workloads.  Index i uses seed SEED_BASE + i.
# --------------------------------------------------------------------------

def mode_sum(shape=(32, 32, 32), m: int = 8, kmax: int = 8, seed: int = SEED_BASE + 1) -> Workload:
    """8 plane waves with k uniform on {-8..8}^3 \\ {0} (32^3, FP64 workload).
    The exact solution is a closed form, because every |k_i| < n_i/2."""
    rng = np.random.default_rng(seed)
    ms = draw_modes(rng, m, kmax)
    return Workload("modes", tuple(shape), eval_modes(ms, shape), modes=ms)


def gaussians16(shape=(256, 256, 256), sigma: float = 0.05, seed: int = SEED_BASE + 2) -> Workload:
    """16 periodised Gaussians of width 0.05, centres uniform, mean removed."""
    rng = np.random.default_rng(seed)
    gs = draw_gaussians(rng, 16, sigma)
    f = eval_gaussians(gs, shape)
    f -= f.mean()
    return Workload("gaussians16", tuple(shape), f, gaussians=gs, mean_subtracted=True)


def sharp_source(shape=(512, 512, 512), seed: int = SEED_BASE + 3) -> Workload:
    """One periodised Gaussian of width 0.01 plus 4 smooth modes with |k| <= 4,
    mean removed (the large-grid workload, 512^3 and 1024^3)."""
    rng = np.random.default_rng(seed)
    gs = draw_gaussians(rng, 1, 0.01)
    ms = draw_modes(rng, 4, 4, max_norm=4.0)
    f = eval_gaussians(gs, shape) + eval_modes(ms, shape)
    f -= f.mean()
    return Workload("sharp_source", tuple(shape), f, modes=ms, gaussians=gs,
                    mean_subtracted=True)


def batch_shapes(count: int = 64, seed: int = SEED_BASE + 4) -> List[Tuple[int, int, int]]:
    """Per-instance grid dims, each axis drawn independently from
    {24, 32, 48, 64, 96, 128, 192, 256}."""
    rng = np.random.default_rng(seed)
    ch = np.array(BATCH_AXIS_CHOICES)
    return [tuple(int(v) for v in rng.choice(ch, size=3)) for _ in range(count)]


def batch_instance(shape, instance: int, seed: int = SEED_BASE + 4) -> Workload:
    """Instance b of the uneven batch: 16 periodised Gaussians with σ ~ U[0.02, 0.1],
    mean removed; seed SEED_BASE + 4 + 1000 + b (disjoint from the shape draw)."""
    rng = np.random.default_rng(seed + 1000 + instance)
    gs = draw_gaussians(rng, 16, (0.02, 0.1))
    f = eval_gaussians(gs, shape)
    f -= f.mean()
    return Workload(f"batch[{instance}]", tuple(shape), f, gaussians=gs, mean_subtracted=True)


def smooth_target(shape=(64, 64, 64), seed: int = SEED_BASE + 5) -> Workload:
    """A smooth target field u_t for the gradient check (8 modes, |k_i| <= 8)."""
    rng = np.random.default_rng(seed)
    ms = draw_modes(rng, 8, 8)
    return Workload("smooth_target", tuple(shape), eval_modes(ms, shape), modes=ms)


def random_field(shape, seed: int) -> np.ndarray:
    """White noise N(0,1) on the grid: the hardest input for a transform
    (every wavenumber excited), used for parity at small sizes."""
    return np.random.default_rng(seed).standard_normal(tuple(shape))


def sphere_layer(shape, alpha: float, R: float = 0.1, centre: float = 0.5, rows=None):
    """The paper's second time-to-solution case (§3, Tables 8-9): the exact
    solution u = exp(-(r/R)^α), r the (minimum-image) distance to the cube's
    centre, a sharp layer at r = R, and its source f = -Δu in closed form:
    with s = (r/R)^α,  -Δu = (α s u / r²)(α + 1 - α s)  (radial Laplacian
    u'' + 2u'/r).  The paper does not state R; R = 0.1 gives the FFT figures
    of its Tables 8 and 9 (Table 9's error at 384³ for α = 40, Table 8's
    grids for α = 10 and 40).  For α >= 10 and R <= 1/4, u and f vanish at the
    cube's faces to far below double precision, so both are smooth periodic
    fields.  Returns (f, u) in float64; rows = (x0, x1) returns only the
    x-slab x0 <= x < x1 (for grids too large to evaluate at once)."""
    axes = []
    for n in shape:
        d = np.arange(n) / n - centre
        d -= np.round(d)  # minimum image
        axes.append(d)
    if rows is not None:
        axes[0] = axes[0][rows[0]:rows[1]]
    r2 = axes[0][:, None, None] ** 2 + axes[1][None, :, None] ** 2 + axes[2][None, None, :] ** 2
    s = (r2 / (R * R)) ** (alpha / 2.0)
    u = np.exp(-s)
    with np.errstate(divide="ignore", invalid="ignore"):
        f = np.where(r2 > 0, alpha * s * u / r2 * (alpha + 1.0 - alpha * s), 0.0)
    return f, u
