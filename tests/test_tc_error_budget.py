"""Error budget of one radix-16 DFT stage on the tensor cores, per operand
format, from a CPU emulation of the rounding the stage performs (CPU only).

The stage computes b = F a for rows a of 16 complex values as a real
[Re a | Im a] (32) × 32×32 product, operands split as x = hi + lo, products
hi·Fhi + hi·Flo + lo·Fhi summed in FP32 (one rounding per K = 16 block, as
the MMAs accumulate).  The emulation fixes the choice of format: BF16
hi/lo leaves a 2^-18 residual of every operand (about 3e-6 per stage, 1e-5
after the eight stages of a 512-point radix-16 plan), FP16 hi/lo with a
power-of-two scale per row keeps 22 bits (within a few percent of FP32
arithmetic).  The kernel's own accuracy is checked on the GPU
(tests/test_gpu_tc.py).
"""
import numpy as np
import pytest


def bf16(x):
    b = np.asarray(x, np.float32).view(np.uint32).astype(np.uint64)
    r = ((b + 0x7FFF + ((b >> 16) & 1)) >> 16) << 16  # round to nearest even
    return r.astype(np.uint32).view(np.float32)


def f16(x):
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float32)


def dft16_real(inverse=False):
    k = np.arange(16)
    ang = 2 * np.pi * np.outer(k, k) / 16
    c, s = np.cos(ang), np.sin(ang)
    fi = s if inverse else -s
    return np.block([[c, -fi], [fi, c]])  # [Re b; Im b] = F [Re a; Im a]


def stage(a, fmt, lolo=False, three_term=False):
    x = np.concatenate([a.real, a.imag], axis=1).astype(np.float32)
    F = dft16_real()
    rnd = bf16 if fmt == "bf16" else f16
    if fmt == "f16":  # largest |component| of each row into [2^14, 2^15)
        m = np.abs(x).max(axis=1, keepdims=True)
        s = np.exp2(14 - np.floor(np.log2(m))).astype(np.float32)
    else:
        s = np.ones((len(x), 1), np.float32)
    xs = x * s
    if three_term:
        a1 = rnd(xs); a2 = rnd(xs - a1); a3 = rnd(xs - a1 - a2)
        F1 = rnd(F); F2 = rnd(F - F1); F3 = rnd(F - F1 - F2)
        prods = [(a1, F1), (a1, F2), (a2, F1), (a1, F3), (a2, F2), (a3, F1)]
    else:
        h = rnd(xs); lo = rnd(xs - h)
        Fh = rnd(F); Fl = rnd(F - Fh)
        prods = [(h, Fh), (h, Fl), (lo, Fh)] + ([(lo, Fl)] if lolo else [])
    acc = np.zeros((len(x), 32))
    for A, B in prods:
        for ks in range(2):
            sl = slice(16 * ks, 16 * ks + 16)
            acc = (acc + A[:, sl].astype(np.float64) @ B[:, sl].T.astype(np.float64)).astype(np.float32)
    y = acc / s
    return y[:, :16] + 1j * y[:, 16:]


def rel(y, ref):
    return float(np.linalg.norm(y - ref) / np.linalg.norm(ref))


@pytest.fixture(scope="module")
def rows():
    rng = np.random.default_rng(16)
    a = (rng.standard_normal((4096, 16)) + 1j * rng.standard_normal((4096, 16))).astype(np.complex64)
    return a, np.fft.fft(a.astype(np.complex128), axis=1)


def test_error_budget_per_format(rows):
    a, ref = rows
    e = {"bf16": rel(stage(a, "bf16"), ref), "bf16_lolo": rel(stage(a, "bf16", lolo=True), ref),
         "bf16_3term": rel(stage(a, "bf16", three_term=True), ref), "f16": rel(stage(a, "f16"), ref)}
    fp32 = rel((a[:, None, :] * np.exp(-2j * np.pi * np.outer(np.arange(16), np.arange(16)) / 16)
                .astype(np.complex64)[None]).sum(-1), ref)
    print({k: f"{v:.2e}" for k, v in e.items()}, f"fp32 {fp32:.2e}")
    # BF16 hi/lo: the 2^-18 operand residual dominates, lo·lo hardly helps
    assert 2e-6 < e["bf16"] < 5e-6 and 2e-6 < e["bf16_lolo"] < e["bf16"]
    # 22 significant bits: FP16 hi/lo (three products) as good as a BF16
    # three-term split (six products), within 30% of FP32 arithmetic
    assert e["f16"] < 1.3 * fp32 and e["bf16_3term"] < 1.3 * fp32


@pytest.mark.parametrize("scale", [1e-30, 1e-8, 1.0, 1e8, 1e30])
def test_row_scale_keeps_fp16_range(rows, scale):
    # without the per-row scale FP16 would overflow (> 65504) or lose the
    # rows to underflow; with it the error is the same at every magnitude
    a, ref = rows
    e = rel(stage(a * scale, "f16"), ref * scale)
    assert e < 1.5e-7, (scale, e)
