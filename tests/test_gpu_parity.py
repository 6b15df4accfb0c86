"""CUDA path vs the FP64 oracle, element by element, through the C ABI.

Tolerances against the oracle solving the same rounded input (tests/tolerances.py):
relative L2 FP64 1e-12, FP32 5e-6; relative ℓ∞ FP64 1e-12, FP32 1e-5.
Wavenumber indexing is compared bit-exactly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import closed_form as cf
from paper_1408_6497_gb300 import Plan, error_norms, poisson_solve
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import TOL, check

pytestmark = pytest.mark.gpu
NP = {"f64": np.float64, "f32": np.float32}


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    oracle.build()


def gpu_solve(f64, prec, batch=1):
    f = f64.astype(NP[prec])
    plan = Plan(f.shape[-3:], dtype=prec, batch=batch)
    ft = torch.from_numpy(np.ascontiguousarray(f).ravel()).cuda()
    u = plan.execute(ft)
    plan.status()
    return u.cpu().numpy().reshape(f.shape), f


SHAPES = [(4, 4, 4), (8, 6, 4), (6, 6, 6), (12, 24, 48), (16, 32, 64), (24, 32, 48), (96, 48, 24),
          (18, 54, 12), (4, 6, 8), (64, 64, 64), (128, 96, 24), (36, 12, 6), (48, 16, 256),
          (2048, 4, 8), (4, 2048, 4), (8, 4, 2048), (162, 8, 18), (32, 32, 1024),
          (96, 48, 128), (24, 8, 256)]


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", SHAPES)
def test_random_field_parity(prec, shape):
    f64 = wl.random_field(shape, seed=100 + sum(shape))
    u, f_in = gpu_solve(f64, prec)
    check(u, oracle.solve(f_in.astype(np.float64)), prec, shape)


@pytest.mark.parametrize("prec,shape", [("f32", (1458, 12, 16)), ("f32", (16, 1458, 8)), ("f64", (16, 1458, 8)),
                                        ("f64", (8, 12, 1458))])
def test_lines_of_1458_points(prec, shape):
    # 2·3^6: six radix-3 stages; 243 threads per line (FP64 x lines of this
    # length are refused at plan creation, the other axes are not)
    f64 = wl.random_field(shape, seed=1458 + sum(shape))
    u, f_in = gpu_solve(f64, prec)
    check(u, oracle.solve(f_in.astype(np.float64)), prec, shape)


# Lines of 256/512/1024 points go through the persistent TMA-fed y/x passes
# in FP32 (column tiles of 32/16/8); 96 and 48 leave a ragged last tile.
TMA_SHAPES = [(256, 512, 96), (512, 256, 32), (1024, 256, 16), (256, 1024, 48), (512, 512, 64),
              (256, 256, 256)]


@pytest.mark.parametrize("shape", TMA_SHAPES)
def test_tma_pass_parity_fp32(shape):
    f64 = wl.random_field(shape, seed=300 + sum(shape))
    u, f_in = gpu_solve(f64, "f32")
    check(u, oracle.solve(f_in.astype(np.float64)), "f32", shape)


def test_tma_pass_batch_fp32():
    shape, B = (256, 256, 32), 3
    f = np.stack([wl.random_field(shape, seed=70 + b) for b in range(B)])
    u, f_in = gpu_solve(f, "f32", batch=B)
    for b in range(B):
        check(u[b], oracle.solve(f_in[b].astype(np.float64)), "f32")


# z rows of 512/1024 points with y lines of 256/512/1024 points take the
# fused z/y cluster passes in FP32 (one plane per cluster, L2 hand-off).
FUSED_SHAPES = [(128, 256, 512), (64, 512, 1024), (32, 1024, 512), (48, 512, 512)]


@pytest.mark.parametrize("shape", FUSED_SHAPES)
def test_fused_zy_parity_fp32(shape, monkeypatch):
    monkeypatch.setenv("PSOLVE_FUSED", "4")
    f64 = wl.random_field(shape, seed=800 + sum(shape))
    plan = Plan(shape, dtype="f32")
    names = [plan.lib.psolve_pass_name(plan.handle, i).decode() for i in range(3)]
    assert names == ["zyfwd", "xdiv", "yzinv"]
    f = torch.from_numpy(f64.astype(np.float32).ravel()).cuda()
    u = plan.execute(f)
    plan.status()
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape))
    check(u.cpu().numpy().reshape(shape), ref, "f32", shape)
    uu = f.clone()
    plan.execute(uu, uu)  # in place
    assert torch.equal(uu, u)


# z rows of 256/512 points with y lines of 256/512 points: the z and y
# transforms of a plane in one 16-block cluster's distributed shared memory
# (three passes through HBM); 4 x-planes leave most clusters idle.
CLUSTER_SHAPES = [(64, 512, 512), (32, 256, 256), (48, 512, 256), (24, 256, 512), (4, 512, 512),
                  (512, 512, 512)]


@pytest.mark.parametrize("shape", CLUSTER_SHAPES)
def test_cluster_zy_parity_fp32(shape, monkeypatch):
    monkeypatch.setenv("PSOLVE_FUSED", "16")
    f64 = wl.random_field(shape, seed=850 + sum(shape))
    plan = Plan(shape, dtype="f32")
    names = [plan.lib.psolve_pass_name(plan.handle, i).decode() for i in range(3)]
    assert names == ["zyfwd", "xdiv", "yzinv"]
    assert plan.launches_per_solve == 3
    f = torch.from_numpy(f64.astype(np.float32).ravel()).cuda()
    u = plan.execute(f)
    plan.status()
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape))
    check(u.cpu().numpy().reshape(shape), ref, "f32", shape)
    uu = f.clone()
    plan.execute(uu, uu)  # in place
    plan.status()
    assert torch.equal(uu, u)


def test_cluster_zy_batch_and_adjoint_fp32(monkeypatch):
    monkeypatch.setenv("PSOLVE_FUSED", "16")
    shape, B = (16, 512, 512), 3
    f = np.stack([wl.random_field(shape, seed=95 + b) for b in range(B)])
    u, f_in = gpu_solve(f, "f32", batch=B)
    for b in range(B):
        check(u[b], oracle.solve(f_in[b].astype(np.float64)), "f32")


def test_cluster_zy_host_buffers(monkeypatch):
    # host-buffer solves of a cluster plan: pinned buffers go through the
    # five-pass path (the cluster kernels read f with bulk copies from device
    # memory only), pageable ones through the staging buffer and the cluster
    monkeypatch.setenv("PSOLVE_FUSED", "16")
    shape = (32, 512, 256)
    f = torch.from_numpy(wl.random_field(shape, seed=96).astype(np.float32).ravel())
    plan = Plan(shape, dtype="f32")
    u_dev = plan.execute(f.cuda()).cpu()
    fp = f.pin_memory()
    up = torch.empty_like(fp).pin_memory()
    plan.execute_host(fp, up)
    ref = oracle.solve(f.numpy().astype(np.float64).reshape(shape))
    check(up.numpy().reshape(shape), ref, "f32")
    u_pg = plan.execute_host(f.numpy())
    assert np.array_equal(u_pg, u_dev.numpy())


def test_fused_zy_batch_fp32(monkeypatch):
    monkeypatch.setenv("PSOLVE_FUSED", "4")
    shape, B = (32, 256, 512), 3
    f = np.stack([wl.random_field(shape, seed=90 + b) for b in range(B)])
    u, f_in = gpu_solve(f, "f32", batch=B)
    for b in range(B):
        check(u[b], oracle.solve(f_in[b].astype(np.float64)), "f32")


# The x-split spectrum layout (rows ordered (x / G, y, x mod G) in the plan's
# own spectrum buffer): forced on shapes that take the bulk z passes and the
# TMA y/x passes, single and uniform-batch plans, in and out of place.
XS_SHAPES = [(256, 256, 512), (512, 256, 1024), (1024, 256, 512), (256, 512, 512)]


@pytest.mark.parametrize("G", ["2", "4", "8"])
@pytest.mark.parametrize("shape", XS_SHAPES)
def test_xsplit_layout_parity_fp32(shape, G, monkeypatch):
    f64 = wl.random_field(shape, seed=900 + sum(shape))
    f = torch.from_numpy(f64.astype(np.float32).ravel()).cuda()
    monkeypatch.setenv("PSOLVE_XSPLIT", "1")
    u_nat = Plan(shape, dtype="f32").execute(f)
    monkeypatch.setenv("PSOLVE_XSPLIT", G)
    free0 = torch.cuda.mem_get_info()[0]
    plan = Plan(shape, dtype="f32")
    # the plan owns a spectrum buffer of the grid's size
    assert free0 - torch.cuda.mem_get_info()[0] >= f.numel() * 4
    u = plan.execute(f)
    plan.status()
    ref = oracle.solve(f.cpu().numpy().astype(np.float64).reshape(shape))
    check(u.cpu().numpy().reshape(shape), ref, "f32")
    # same butterflies in another memory order: identical results
    assert torch.equal(u, u_nat)
    uu = f.clone()
    plan.execute(uu, uu)  # in place: f and u are the same array
    assert torch.equal(uu, u)


def test_xsplit_layout_batch_fp32(monkeypatch):
    monkeypatch.setenv("PSOLVE_XSPLIT", "4")
    shape, B = (256, 256, 512), 3
    f = np.stack([wl.random_field(shape, seed=60 + b) for b in range(B)])
    u, f_in = gpu_solve(f, "f32", batch=B)
    for b in range(B):
        check(u[b], oracle.solve(f_in[b].astype(np.float64)), "f32")


def test_config1_fp64_mode_sum_closed_form():
    w = wl.mode_sum()
    u, _ = gpu_solve(w.f, "f64")
    ref = oracle.solve(w.f)
    exact = cf.mode_sum_u(w.modes.k, w.modes.a, w.modes.phi, w.shape)
    check(u, ref, "f64")
    check(u, exact, "f64")


def test_config2_fp32_gaussians_256():
    w = wl.gaussians16()
    u, f_in = gpu_solve(w.f, "f32")
    ref = oracle.solve(f_in.astype(np.float64))
    err, linf = check(u, ref, "f32", "256^3 gaussians")
    print(f"256^3 gaussians FP32 rel-L2 {err:.3e} rel-linf {linf:.3e}")


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("shape", [(8, 8, 8), (12, 6, 16)])
def test_single_modes_and_nyquist(prec, shape):
    nx, ny, nz = shape
    x = np.arange(nx)[:, None, None] / nx
    y = np.arange(ny)[None, :, None] / ny
    z = np.arange(nz)[None, None, :] / nz
    ks = [(1, 2, 1), (-1, 2, -1), (1, -2, -1), (nx // 2, 0, 0), (0, ny // 2, 0), (0, 0, nz // 2),
          (nx // 2, ny // 2, nz // 2), (1, ny // 2, nz // 2), (0, 0, 1), (2, 0, nz // 2)]
    for k in ks:
        for trig in (np.cos, np.sin):
            f = trig(2 * np.pi * (k[0] * x + k[1] * y + k[2] * z))
            if np.abs(f).max() < 0.5:
                continue
            u, _ = gpu_solve(f, prec)
            exact = f / (4 * np.pi ** 2 * (k[0] ** 2 + k[1] ** 2 + k[2] ** 2))
            assert np.abs(u - exact).max() <= 10 * TOL[prec] * np.abs(exact).max(), (k, trig)


@pytest.mark.parametrize("shape", [(8, 8, 8), (24, 12, 48), (6, 12, 4)])
def test_kvec_bit_exact(shape):
    plan = Plan(shape, dtype="f32")
    k = plan.debug_kvec(0)
    nx, ny, nz = shape
    kx, ky, kz = oracle.kvec(nx), oracle.kvec(ny), oracle.kvec(nz)
    H = nz // 2 + 1
    np.testing.assert_array_equal(k[..., 0], np.broadcast_to(kx[:, None, None], (nx, ny, H)))
    np.testing.assert_array_equal(k[..., 1], np.broadcast_to(ky[None, :, None], (nx, ny, H)))
    np.testing.assert_array_equal(k[..., 2], np.broadcast_to(kz[None, None, :H], (nx, ny, H)))


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_in_place(prec):
    shape = (16, 24, 12)
    f64 = wl.random_field(shape, seed=7)
    plan = Plan(shape, dtype=prec)
    ft = torch.from_numpy(f64.astype(NP[prec]).ravel()).cuda()
    ref = plan.execute(ft.clone())
    plan.execute(ft, ft)
    assert torch.equal(ft, ref)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_uniform_batch(prec):
    shape, B = (12, 16, 24), 3
    fs = [wl.random_field(shape, seed=40 + b) for b in range(B)]
    f = np.stack(fs)
    u, f_in = gpu_solve(f, prec, batch=B)
    for b in range(B):
        check(u[b], oracle.solve(f_in[b].astype(np.float64)), prec)


@pytest.mark.parametrize("prec", ["f64", "f32"])
def test_uneven_batch(prec):
    shapes = wl.batch_shapes(8)
    plan = Plan(dtype=prec, shapes=shapes)
    flat = plan.empty()
    fs = []
    for b, s in enumerate(shapes):
        w = wl.batch_instance(s, b)
        fs.append(w.f.astype(NP[prec]))
        plan.view(flat, b).copy_(torch.from_numpy(fs[-1]))
    u = plan.execute(flat)
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs[b].astype(np.float64))
        check(plan.view(u, b).cpu().numpy(), ref, prec, s)


def test_execute_host_matches_device():
    shape = (32, 16, 48)
    f = wl.random_field(shape, seed=12).astype(np.float32)
    plan = Plan(shape, dtype="f32")
    u_dev = plan.execute(torch.from_numpy(f.ravel()).cuda()).cpu().numpy()
    u_host = plan.execute_host(f.ravel())
    np.testing.assert_array_equal(u_dev, u_host)


@pytest.mark.parametrize("prec,shape", [("f32", (32, 16, 48)), ("f32", (128, 256, 512)), ("f64", (24, 24, 32))])
def test_execute_host_pinned_zero_copy(prec, shape, monkeypatch):
    """Pinned buffers take the path where the first pass reads f and the last
    writes u across the host link; it must equal the device solve."""
    f = torch.from_numpy(wl.random_field(shape, seed=13).astype(NP[prec]).ravel()).pin_memory()
    u = torch.empty_like(f).pin_memory()
    plan = Plan(shape, dtype=prec)
    u_dev = plan.execute(f.cuda()).cpu()
    plan.execute_host(f, u)
    assert torch.equal(u, u_dev)
    monkeypatch.setenv("PSOLVE_ZERO_COPY", "0")
    u2 = torch.empty_like(f).pin_memory()
    plan.execute_host(f, u2)
    assert torch.equal(u2, u_dev)


def test_execute_host_async_pipelined():
    shape = (64, 128, 256)
    plan = Plan(shape, dtype="f32")
    fs = [torch.from_numpy(wl.random_field(shape, seed=60 + k).astype(np.float32).ravel()).pin_memory()
          for k in range(4)]
    us = [torch.empty_like(f).pin_memory() for f in fs]
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    for k in range(4):
        plan.execute_host_async(fs[k], us[k], streams[k % 2])
    torch.cuda.synchronize()
    for k in range(4):
        assert torch.equal(us[k], plan.execute(fs[k].cuda()).cpu())


def test_adjoint_symmetry_and_autograd_fp64():
    shape = (16, 12, 8)
    x = torch.from_numpy(wl.random_field(shape, seed=1)).cuda()
    y = torch.from_numpy(wl.random_field(shape, seed=2)).cuda()
    plan = Plan(shape, dtype="f64")
    ax = plan.execute(x.ravel())
    ay = plan.adjoint(y.ravel())
    lhs = float((ax * y.ravel()).sum())
    rhs = float((x.ravel() * ay).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)


def test_gradient_64_fp64_vs_oracle_and_fd():
    shape = (64, 64, 64)
    f64 = wl.sharp_source(shape).f
    ut = wl.smooth_target(shape).f * 1e-3
    f = torch.from_numpy(f64).cuda().requires_grad_(True)
    target = torch.from_numpy(ut).cuda()
    u = poisson_solve(f)
    loss = 0.5 * ((u - target) ** 2).sum()
    loss.backward()
    g_or = oracle.gradient(f64, ut)
    check(f.grad.cpu().numpy(), g_or, "f64")

    def L(v):
        with torch.no_grad():
            r = poisson_solve(v) - target
            return 0.5 * float((r * r).sum())

    rng = np.random.default_rng(3)
    h = 1e-4
    for _ in range(3):
        d = torch.from_numpy(rng.standard_normal(shape)).cuda()
        fd = (L(f.detach() + h * d) - L(f.detach() - h * d)) / (2 * h)
        an = float((f.grad * d).sum())
        assert abs(fd - an) <= 1e-6 * abs(an)


def test_error_norms_kernel():
    a = torch.randn(1000, dtype=torch.float64, device="cuda")
    b = a + 1e-3 * torch.randn(1000, dtype=torch.float64, device="cuda")
    l2, linf = error_norms(b, a)
    an, bn = a.cpu().numpy(), b.cpu().numpy()
    assert l2 == pytest.approx(oracle.rel_l2(bn, an), rel=1e-12)
    assert linf == pytest.approx(oracle.rel_linf(bn, an), rel=1e-12)


def test_argument_errors_on_device():
    from paper_1408_6497_gb300 import _lib
    plan = Plan((8, 8, 8), dtype="f32")
    buf = torch.zeros(2 * 512 + 8, dtype=torch.float32, device="cuda")
    lib = _lib.load()
    base = buf.data_ptr()
    # misaligned pointer
    assert lib.psolve_execute(plan.handle, base + 4, base + 4096, None) == 1
    # partial overlap of f and u
    assert lib.psolve_execute(plan.handle, base, base + 64, None) == 1
    # exact aliasing is allowed
    assert lib.psolve_execute(plan.handle, base, base, None) == 0
    torch.cuda.synchronize()


def test_pass_profiling_every_kth_solve():
    plan = Plan((64, 48, 32), dtype="f32")
    f = torch.randn(64 * 48 * 32, device="cuda")
    u = torch.empty_like(f)
    plan.set_profiling(3)
    for _ in range(7):
        plan.execute(f, u)
    ms, nsol = plan.pass_times()
    assert nsol == 3  # solves 0, 3 and 6
    assert list(ms) == ["zfwd", "yfwd", "xdiv", "yinv", "zinv"] and all(v > 0 for v in ms.values())
    plan.set_profiling(0)
    plan.execute(f, u)
    assert plan.pass_times()[1] == 0
    with pytest.raises(Exception):
        plan.set_profiling(-1)
