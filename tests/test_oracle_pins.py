"""Pins of the FP64 oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle — a dropped
factor of 4π², a wrong twiddle sign, a transposed axis, an off-by-one
wavenumber, a lost Nyquist term — fails at least one of them:
  * brute-force Kronecker DFT matrices built here with numpy (4^3 .. 8^3);
  * closed forms: plane-wave sums and the paper's test case 1 (§3, Table 7);
  * numpy.fft as an independent library;
  * Parseval, Hermitian symmetry, zero mean, linearity, the spectral
    Laplacian round trip, and a finite-difference check of the gradient.
"""
import os

import numpy as np
import pytest

from oracle import closed_form as cf
from paper_1408_6497_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dft_matrix(n, sign=-1):
    j = np.arange(n)
    return np.exp(sign * 2j * np.pi * np.outer(j, j) / n)


def signed_k(n):
    """Independent statement of the wavenumber reading: j for j <= n/2,
    j - n otherwise (Nyquist +n/2)."""
    j = np.arange(n)
    return np.where(2 * j <= n, j, j - n)


def brute_force_solve(f):
    nx, ny, nz = f.shape
    F = np.kron(dft_matrix(nx), np.kron(dft_matrix(ny), dft_matrix(nz)))
    Fi = np.kron(dft_matrix(nx, +1), np.kron(dft_matrix(ny, +1), dft_matrix(nz, +1)))
    kx, ky, kz = signed_k(nx), signed_k(ny), signed_k(nz)
    k2 = (kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2).ravel()
    d = np.zeros(k2.shape)
    d[k2 > 0] = 1.0 / (4.0 * np.pi ** 2 * k2[k2 > 0])
    u = Fi @ (d * (F @ f.ravel())) / f.size
    return u.real.reshape(f.shape), F


SMALL = [(4, 4, 4), (6, 4, 8), (8, 8, 8), (4, 6, 6), (3, 5, 4), (8, 6, 2)]


@pytest.mark.parametrize("shape", SMALL)
@pytest.mark.parametrize("direct", [True, False])
def test_bruteforce_kronecker(oracle_mod, shape, direct):
    f = wl.random_field(shape, seed=11 + sum(shape))
    u_bf, F = brute_force_solve(f)
    u = oracle_mod.solve(f, direct=direct)
    assert oracle_mod.rel_l2(u, u_bf) < 1e-13
    spec = oracle_mod.dft3d(f, direct=direct)
    ref = (F @ f.ravel()).reshape(shape)
    assert np.abs(spec - ref).max() < 1e-12 * np.abs(ref).max()
    back = oracle_mod.dft3d(spec, inverse=True, direct=direct) / f.size
    assert np.abs(back - f).max() < 1e-13 * np.abs(f).max()


def test_mode_sum_closed_form(oracle_mod):
    w = wl.mode_sum()  # 32^3, 8 modes, |k_i| <= 8 < 16
    u = oracle_mod.solve(w.f)
    u_ex = cf.mode_sum_u(w.modes.k, w.modes.a, w.modes.phi, w.shape)
    assert oracle_mod.rel_l2(u, u_ex) < 1e-13
    # the generator's factorised plane waves equal the direct sin evaluation
    f_ex = cf.mode_sum_f(w.modes.k, w.modes.a, w.modes.phi, w.shape)
    assert np.abs(w.f - f_ex).max() < 1e-12


@pytest.mark.parametrize("shape", [(16, 24, 12), (18, 12, 36)])
def test_mode_sum_closed_form_noncubic(oracle_mod, shape):
    rng = np.random.default_rng(5)
    lim = [n // 2 - 1 for n in shape]
    k = np.array([[rng.integers(-l, l + 1) for l in lim] for _ in range(6)])
    k = k[np.any(k != 0, axis=1)]
    a, phi = rng.standard_normal(len(k)), rng.uniform(0, 2 * np.pi, len(k))
    f = cf.mode_sum_f(k, a, phi, shape)
    for direct in (False, True):
        u = oracle_mod.solve(f, direct=direct)
        assert oracle_mod.rel_l2(u, cf.mode_sum_u(k, a, phi, shape)) < 1e-12


def _table7_rows():
    rows = []
    with open(os.path.join(GOLDEN, "paper_table7_fft.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                p, k, L = (int(v) for v in line.split())
                rows.append((p, k, L))
    return rows


@pytest.mark.parametrize("row", [r for r in _table7_rows() if r[2] <= 7])
def test_paper_case1_machine_precision(oracle_mod, row):
    """Table 7: at n = 2^L the FFT resolves test case 1 with wavenumber k to
    machine accuracy (rows with n <= 128 run here)."""
    _, kw, L = row
    n = 2 ** L
    shape = (n, n, n)
    u_ex = cf.paper_case1_u(kw, shape)
    u = oracle_mod.solve(cf.paper_case1_f(kw, shape))
    assert oracle_mod.rel_linf(u, u_ex) < 1e-12


def test_table7_rows_need_n_above_2k():
    """The reading adopted for '2k points per dimension': sin(2πk x) sampled
    at n = 2k vanishes identically, so each row of Table 7 has n > 2k."""
    for _, kw, L in _table7_rows():
        assert 2 ** L > 2 * kw
        assert np.abs(cf.paper_case1_u(kw, (2 * kw, 2 * kw, 2 * kw))).max() < 1e-12


@pytest.mark.parametrize("shape", [(8, 12, 16), (24, 32, 48), (32, 32, 32), (18, 54, 12), (96, 24, 48)])
def test_numpy_fft_crosscheck(oracle_mod, shape):
    f = wl.random_field(shape, seed=3 + shape[0])
    F = np.fft.rfftn(f)
    kx = np.fft.fftfreq(shape[0]) * shape[0]
    ky = np.fft.fftfreq(shape[1]) * shape[1]
    kz = np.fft.rfftfreq(shape[2]) * shape[2]
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    k2[0, 0, 0] = np.inf
    u_np = np.fft.irfftn(F / (4 * np.pi ** 2 * k2), s=shape, axes=(0, 1, 2))
    assert oracle_mod.rel_l2(oracle_mod.solve(f), u_np) < 1e-13


@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 16)])
def test_parseval_and_hermitian(oracle_mod, shape):
    f = wl.random_field(shape, seed=21)
    F = oracle_mod.dft3d(f)
    assert abs((f ** 2).sum() - (np.abs(F) ** 2).sum() / f.size) < 1e-12 * (f ** 2).sum()
    nx, ny, nz = shape
    ix, iy, iz = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij")
    mirror = F[(-ix) % nx, (-iy) % ny, (-iz) % nz]
    assert np.abs(mirror - np.conj(F)).max() < 1e-12 * np.abs(F).max()


def test_zero_mean_and_mean_invariance(oracle_mod):
    f = wl.random_field((12, 16, 8), seed=4)
    u = oracle_mod.solve(f)
    assert abs(u.mean()) < 1e-16 * np.abs(u).max() * 10
    u2 = oracle_mod.solve(f + 3.25)
    assert np.abs(u2 - u).max() < 1e-14 * np.abs(u).max()


def test_linearity(oracle_mod):
    f = wl.random_field((8, 12, 6), seed=8)
    g = wl.random_field((8, 12, 6), seed=9)
    lhs = oracle_mod.solve(2.5 * f - 0.75 * g)
    rhs = 2.5 * oracle_mod.solve(f) - 0.75 * oracle_mod.solve(g)
    assert np.abs(lhs - rhs).max() < 1e-13 * np.abs(rhs).max()


@pytest.mark.parametrize("shape", [(16, 8, 12), (6, 6, 6)])
def test_spectral_laplacian_roundtrip(oracle_mod, shape):
    """-Δ applied spectrally (×4π²|k|², k from this file) to u gives f - mean f."""
    f = wl.random_field(shape, seed=17)
    u = oracle_mod.solve(f)
    kx, ky, kz = (signed_k(n) for n in shape)
    k2 = kx[:, None, None] ** 2 + ky[None, :, None] ** 2 + kz[None, None, :] ** 2
    back = oracle_mod.dft3d(oracle_mod.dft3d(u) * (4 * np.pi ** 2 * k2), inverse=True).real / f.size
    assert np.abs(back - (f - f.mean())).max() < 1e-12 * np.abs(f).max()


@pytest.mark.parametrize("shape", [(8, 8, 8), (6, 10, 4)])
def test_single_modes_every_octant_and_nyquist(oracle_mod, shape):
    """cos(2π k·x) for k in every sign octant, including Nyquist components,
    solves to itself over 4π²|k|² (the Nyquist mode is kept, k² = (n/2)²)."""
    nx, ny, nz = shape
    x = np.arange(nx)[:, None, None] / nx
    y = np.arange(ny)[None, :, None] / ny
    z = np.arange(nz)[None, None, :] / nz
    cases = []
    for sx in (1, -1):
        for sy in (1, -1):
            for sz in (1, -1):
                cases.append((sx * 1, sy * 2, sz * 1))
    cases += [(nx // 2, 0, 0), (0, ny // 2, 0), (0, 0, nz // 2), (nx // 2, ny // 2, nz // 2), (1, ny // 2, 1)]
    for k in cases:
        f = np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z))
        u = oracle_mod.solve(f)
        k2 = k[0] ** 2 + k[1] ** 2 + k[2] ** 2
        assert np.abs(u - f / (4 * np.pi ** 2 * k2)).max() < 1e-14, k


@pytest.mark.parametrize("n", [2, 3, 4, 6, 8, 9, 12, 16, 24, 96])
def test_kvec_convention(oracle_mod, n):
    k = oracle_mod.kvec(n)
    ref = np.rint(np.fft.fftfreq(n) * n).astype(np.int64)
    if n % 2 == 0:
        assert k[n // 2] == n // 2 and ref[n // 2] == -(n // 2)
        ref[n // 2] = n // 2
    np.testing.assert_array_equal(k, ref)
    np.testing.assert_array_equal(k ** 2, signed_k(n) ** 2)


def test_symbol_inverse_values(oracle_mod):
    d = oracle_mod.symbol_inverse((4, 6, 8))
    assert d[0, 0, 0] == 0.0
    assert d[1, 0, 0] == pytest.approx(1 / (4 * np.pi ** 2))
    assert d[3, 5, 7] == pytest.approx(1 / (4 * np.pi ** 2 * 3))      # k = (-1,-1,-1)
    assert d[2, 3, 4] == pytest.approx(1 / (4 * np.pi ** 2 * (4 + 9 + 16)))


def test_gradient_finite_differences(oracle_mod):
    """∇_f ½‖A f − u_t‖² = A (A f − u_t), checked by central differences."""
    shape = (8, 6, 8)
    f = wl.random_field(shape, seed=31)
    ut = 1e-2 * wl.random_field(shape, seed=32)
    g = oracle_mod.gradient(f, ut)

    def loss(v):
        r = oracle_mod.solve(v) - ut
        return 0.5 * float((r * r).sum())

    rng = np.random.default_rng(33)
    h = 1e-3
    for _ in range(4):
        d = rng.standard_normal(shape)
        fd = (loss(f + h * d) - loss(f - h * d)) / (2 * h)
        assert fd == pytest.approx(float((g * d).sum()), rel=1e-8, abs=1e-14)


def test_direct_and_recursive_agree_with_prime_factor(oracle_mod):
    f = wl.random_field((10, 12, 14), seed=41)  # 5 and 7 go to the direct fallback
    a = oracle_mod.solve(f, direct=True)
    b = oracle_mod.solve(f, direct=False)
    assert oracle_mod.rel_l2(b, a) < 1e-13


def test_imaginary_part_vanishes(oracle_mod):
    f = wl.random_field((16, 12, 10), seed=5)
    _, mi = oracle_mod.solve(f, return_imag=True)
    assert mi < 1e-15


# ------------------------------------------------- other operators (widening)
def _neg_fd_laplacian(u):
    """The 7-point stencil −Σ_axes (u[i+1] − 2u[i] + u[i−1]) / h², h = 1/n,
    periodic, written out with numpy rolls (independent of any transform)."""
    out = np.zeros_like(u)
    for ax in range(3):
        n = u.shape[ax]
        out -= (np.roll(u, 1, ax) - 2.0 * u + np.roll(u, -1, ax)) * float(n * n)
    return out


@pytest.mark.parametrize("shape", [(8, 6, 4), (12, 16, 6), (9, 8, 10), (6, 6, 6)])
def test_fd_operator_solves_the_7_point_stencil(oracle_mod, shape):
    f = np.random.default_rng(sum(shape)).standard_normal(shape)
    f -= f.mean()
    u = oracle_mod.solve(f, op="fd")
    r = _neg_fd_laplacian(u) - f
    assert np.abs(r).max() <= 1e-11 * np.abs(f).max()
    assert abs(u.mean()) <= 1e-13 * np.abs(u).max()


def test_fd_operator_limit_is_the_spectral_one(oracle_mod):
    # a smooth mode on a fine grid: the stencil's eigenvalue approaches 4π²|k|²
    shape = (64, 64, 64)
    x = np.arange(64) / 64.0
    f = np.sin(2 * np.pi * x)[:, None, None] * np.ones(shape)
    u_fd, u_sp = oracle_mod.solve(f, op="fd"), oracle_mod.solve(f)
    lam = 4 * 64 ** 2 * np.sin(np.pi / 64) ** 2
    assert np.allclose(u_fd, f / lam, rtol=0, atol=1e-13)
    assert 0 < oracle_mod.rel_l2(u_fd, u_sp) < 1e-3  # O(h²) apart


@pytest.mark.parametrize("n,k", [(2048, 1), (2048, 3), (1458, 1), (1944, 2)])
def test_fd_lowest_modes_of_fine_grids_to_full_precision(oracle_mod, n, k):
    # A single mode cos(2πkx) of a fine grid is an eigenvector of the stencil
    # with eigenvalue (2/h²)(1 − cos 2πk/n); evaluated in 40-digit arithmetic
    # (mpmath, independent of the oracle), u = f/λ must hold to FP64 rounding.
    # These are the modes a solve's u is made of, and the ones where the
    # cosine form of λ loses digits to cancellation in FP64.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    lam = float(2 * mp.mpf(n) ** 2 * (1 - mp.cos(2 * mp.pi * k / n)))
    x = np.arange(n) / n
    f = np.cos(2 * np.pi * k * x)[:, None, None] * np.ones((n, 4, 6))
    u = oracle_mod.solve(f, op="fd")
    assert np.abs(u - f / lam).max() <= 1e-14 * np.abs(f / lam).max()


@pytest.mark.parametrize("c", [0.5, 3.7, 1e3])
def test_helmholtz_modes_and_constant(oracle_mod, c):
    shape = (8, 12, 6)
    x = np.arange(8)[:, None, None] / 8
    y = np.arange(12)[None, :, None] / 12
    z = np.arange(6)[None, None, :] / 6
    for k in [(1, 2, 0), (0, 0, 3), (2, -5, 1), (4, 6, 3)]:
        f = np.cos(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z)) + 0 * x * y * z
        u = oracle_mod.solve(f, op="helmholtz", c=c)
        expect = f / (4 * np.pi ** 2 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2) + c)
        assert np.abs(u - expect).max() <= 1e-13 * np.abs(f).max()
    u = oracle_mod.solve(np.full(shape, 2.5), op="helmholtz", c=c)
    assert np.allclose(u, 2.5 / c, rtol=1e-14, atol=0)  # the mean is kept


def test_operators_are_self_adjoint(oracle_mod):
    rng = np.random.default_rng(5)
    shape = (6, 8, 10)
    a, b = rng.standard_normal(shape), rng.standard_normal(shape)
    for op, c in (("helmholtz", 2.0), ("fd", 0.0)):
        lhs = float((oracle_mod.solve(a, op=op, c=c) * b).sum())
        rhs = float((a * oracle_mod.solve(b, op=op, c=c)).sum())
        assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1.0)
