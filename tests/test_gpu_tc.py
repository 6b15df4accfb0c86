"""Tensor-core (tcgen05) radix-16 stage against a reference DFT."""
import numpy as np
import pytest
import torch

from paper_1408_6497_gb300 import _lib

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
def test_tc_dft16_matches_reference(lib, nb, inverse):
    rng = np.random.default_rng(nb + inverse)
    x = (rng.standard_normal((nb, 16)) + 1j * rng.standard_normal((nb, 16))).astype(np.complex64)
    xin = torch.from_numpy(x.view(np.float32).copy()).cuda()
    out = torch.zeros_like(xin)
    rc = lib.psolve_debug_tc_dft16(xin.data_ptr(), out.data_ptr(), nb, inverse,
                                   torch.cuda.current_stream().cuda_stream)
    assert rc == 0, _lib.STATUS.get(rc, rc)
    y = out.cpu().numpy().view(np.complex64).reshape(nb, 16).astype(np.complex128)
    xd = x.astype(np.complex128)
    ref = np.fft.ifft(xd, axis=1) * 16 if inverse else np.fft.fft(xd, axis=1)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    # BF16 hi/lo operands, FP32 accumulation: ~2^-18 per product
    assert err < 1e-5, err
    assert err > 1e-9  # it really went through BF16 (not an FP32 copy)


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


@pytest.mark.parametrize("shape", [(256, 256, 64), (512, 256, 32), (256, 1024, 32), (1024, 256, 64)])
def test_tc_solve_parity(lib, shape):
    oracle.build()
    f64 = wl.random_field(shape, seed=700 + sum(shape))
    u, f_in, names = _solve(shape, "f32_tc", f64)
    assert "yfwd_tc" in names and "xdiv_tc" in names and "yinv_tc" in names
    err = oracle.rel_l2(u, oracle.solve(f_in.astype(np.float64)))
    assert err <= 1e-5, (shape, err)


def test_tc_solve_512_sharp_source_vs_oracle_and_fp32(lib):
    """The tensor-core workload: 512^3 sharp source, rel-L2 <= 1e-5 against
    the FP64 oracle, reported next to the plain FP32 path's error."""
    oracle.build()
    shape = (512, 512, 512)
    w = wl.sharp_source(shape)
    u_tc, f_in, names = _solve(shape, "f32_tc", w.f)
    u_32, _, _ = _solve(shape, "f32", w.f)
    ref = oracle.solve(f_in.astype(np.float64))
    e_tc, e_32 = oracle.rel_l2(u_tc, ref), oracle.rel_l2(u_32, ref)
    print(f"512^3 sharp source rel-L2: tensor-core {e_tc:.3e}, FP32 {e_32:.3e}; passes {names}")
    assert e_tc <= 1e-5
    assert e_32 <= 5e-6


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
    err = oracle.rel_l2(u, oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape)))
    assert 1e-7 < err <= 1e-5  # tensor-core accuracy, not an FP32 result


@pytest.mark.parametrize("cfg", ["1,1", "0,0", "3,3", "4,4", "3,4"])
def test_tc_512_line_configurations(lib, monkeypatch, cfg):
    """Every tensor-core variant of the 512-point y and x passes: plans of
    radix-16 stages (16 points per thread: configurations 0, 1) and the
    32 × 16 plan with its radix-16 stage on the tensor cores per warpgroup
    (32 points per thread: 3 with one warpgroup per block, 4 with two)."""
    monkeypatch.setenv("PSOLVE_TMA_NARROW", cfg)
    oracle.build()
    shape = (512, 512, 32)
    # the tensor-core workload's source (sharp Gaussian + low modes), for which
    # the 1e-5 bound is stated; white noise through the eight radix-16 stages
    # of the 16-point-per-thread plans lands at about 1e-5 itself
    f64 = wl.sharp_source(shape).f
    u, f_in, names = _solve(shape, "f32_tc", f64)
    assert names == ["zfwd", "yfwd_tc", "xdiv_tc", "yinv_tc", "zinv"]
    err = oracle.rel_l2(u, oracle.solve(f_in.astype(np.float64)))
    assert 1e-7 < err <= 1e-5, (cfg, err)
