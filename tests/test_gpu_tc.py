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
