"""Tensor-core (tcgen05) radix-16 stage against a reference DFT, and the
tensor-core solve path against the FP64 oracle (rel-L2 ≤ 1e-5, rel-ℓ∞ ≤ 2e-5)."""
import numpy as np
import pytest
import torch

from paper_1408_6497_gb300 import _lib

from .tolerances import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    return _lib.load()


@pytest.mark.parametrize("nb", [1, 128, 256, 1000, 4096])
@pytest.mark.parametrize("inverse", [0, 1])
@pytest.mark.parametrize("scale", [1.0, 1e-25, 1e6, 1e25])
def test_tc_dft16_matches_reference(lib, nb, inverse, scale):
    """One radix-16 stage on the tensor cores: FP16 hi/lo operands with a
    power-of-two scale per row.  The per-row scale keeps the error at the
    FP32 level whatever the magnitude of the rows (FP16 alone would
    overflow above 65504 and lose everything below 2^-24)."""
    rng = np.random.default_rng(nb + inverse)
    x = (rng.standard_normal((nb, 16)) + 1j * rng.standard_normal((nb, 16)))
    # rows of very different magnitudes in one launch
    x *= scale * np.exp2(rng.integers(-20, 21, size=(nb, 1)))
    x = x.astype(np.complex64)
    xin = torch.from_numpy(x.view(np.float32).copy()).cuda()
    out = torch.zeros_like(xin)
    rc = lib.psolve_debug_tc_dft16(xin.data_ptr(), out.data_ptr(), nb, inverse,
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0, _lib.STATUS.get(rc, rc)
    y = out.cpu().numpy().view(np.complex64).reshape(nb, 16).astype(np.complex128)
    xd = x.astype(np.complex128)
    ref = np.fft.ifft(xd, axis=1) * 16 if inverse else np.fft.fft(xd, axis=1)
    # per row, relative to that row's norm (rows differ by up to 2^40)
    err = np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)
    # 22-bit operands, FP32 accumulation: the CPU emulation of the format
    # gives 7.6e-8 for unit rows (FP32 arithmetic: 6.3e-8)
    assert float(np.sqrt(np.mean(err ** 2))) < 3e-7, err.max()
    assert err.max() < 1e-6


# ---------------------------------------------------------------- solves
import oracle  # noqa: E402
from paper_1408_6497_gb300 import Plan  # noqa: E402
from paper_1408_6497_gb300 import workloads as wl  # noqa: E402


def _solve(shape, prec, f64):
    plan = Plan(shape, dtype=prec)
    f = torch.from_numpy(f64.astype(np.float32).ravel()).cuda()
    u = plan.execute(f)
    plan.status()
    names = [plan.lib.psolve_pass_name(plan.handle, i).decode() for i in range(5)]
    return u.cpu().numpy().reshape(shape), f.cpu().numpy().reshape(shape), names


@pytest.mark.parametrize("shape", [(256, 256, 64), (512, 256, 32), (256, 1024, 32), (1024, 256, 64),
                                   (1024, 1024, 16)])
def test_tc_solve_parity(lib, shape):
    """White noise (every wavenumber excited) through the tensor-core passes
    of 256-, 512- and 1024-point lines."""
    oracle.build()
    f64 = wl.random_field(shape, seed=700 + sum(shape))
    u, f_in, names = _solve(shape, "f32_tc", f64)
    assert "yfwd_tc" in names and "xdiv_tc" in names and "yinv_tc" in names
    check(u, oracle.solve(f_in.astype(np.float64)), "f32_tc", shape)


def test_tc_solve_512_sharp_source_vs_oracle_and_fp32(lib):
    """The tensor-core workload: 512^3 sharp source against the FP64 oracle,
    reported next to the plain FP32 path's error."""
    oracle.build()
    shape = (512, 512, 512)
    w = wl.sharp_source(shape)
    u_tc, f_in, names = _solve(shape, "f32_tc", w.f)
    u_32, _, _ = _solve(shape, "f32", w.f)
    ref = oracle.solve(f_in.astype(np.float64))
    e_tc = check(u_tc, ref, "f32_tc", "512^3 tensor cores")
    e_32 = check(u_32, ref, "f32", "512^3 FP32")
    print(f"512^3 sharp source (rel-L2, rel-linf): tensor-core {e_tc}, FP32 {e_32}; passes {names}")


def test_tc_solve_512_white_noise(lib):
    """512^3 white noise through the default tensor-core plan."""
    oracle.build()
    shape = (512, 512, 512)
    f64 = wl.random_field(shape, seed=5120)
    u, f_in, names = _solve(shape, "f32_tc", f64)
    assert names == ["zfwd", "yfwd_tc", "xdiv_tc", "yinv_tc", "zinv"]
    e = check(u, oracle.solve(f_in.astype(np.float64)), "f32_tc", "512^3 white noise")
    print(f"512^3 white noise tensor-core (rel-L2, rel-linf) {e}")


def test_tc_plan_stays_on_tensor_cores_after_autotune(lib, tmp_path, monkeypatch):
    monkeypatch.setenv("PSOLVE_TUNE_CACHE", str(tmp_path / "tune.txt"))
    oracle.build()
    shape = (256, 512, 64)
    plan = Plan(shape, dtype="f32_tc")
    plan.autotune()
    names = [plan.lib.psolve_pass_name(plan.handle, i).decode() for i in range(5)]
    assert names == ["zfwd", "yfwd_tc", "xdiv_tc", "yinv_tc", "zinv"]
    f64 = wl.random_field(shape, seed=3)
    f = torch.from_numpy(f64.astype(np.float32).ravel()).cuda()
    u = plan.execute(f).cpu().numpy().reshape(shape)
    check(u, oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape)), "f32_tc", shape)


@pytest.mark.parametrize("cfg", ["1,1", "0,0", "3,3", "4,4", "3,4"])
def test_tc_512_line_configurations(lib, monkeypatch, cfg):
    """Every tensor-core variant of the 512-point y and x passes on white
    noise: plans of radix-16 stages (16 points per thread: configurations
    0, 1; eight tensor-core stages per solve) and the 32 × 16 plan with its
    radix-16 stage on the tensor cores per warpgroup (32 points per thread:
    3 with one warpgroup per block, 4 with two)."""
    monkeypatch.setenv("PSOLVE_TMA_NARROW", cfg)
    oracle.build()
    shape = (512, 512, 32)
    f64 = wl.random_field(shape, seed=512 + int(cfg[0]) * 10 + int(cfg[2]))
    u, f_in, names = _solve(shape, "f32_tc", f64)
    assert names == ["zfwd", "yfwd_tc", "xdiv_tc", "yinv_tc", "zinv"]
    check(u, oracle.solve(f_in.astype(np.float64)), "f32_tc", cfg)
