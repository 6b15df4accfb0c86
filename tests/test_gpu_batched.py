"""Batched solves of unequal grids: one persistent launch from a CUDA graph.

64 right-hand sides with every axis drawn from {24, 32, 48, 64, 96, 128,
192, 256} (radix-2/3, non-cubic), each compared with its own FP64 oracle
solve; graph replays with new data and new buffers; and the bounded wait of
the persistent kernel, made to run out on purpose, which must come back as
PSOLVE_ERR_TIMEOUT with the context still usable.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1408_6497_gb300 import Plan, _lib
from paper_1408_6497_gb300 import workloads as wl

from .tolerances import check

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1408_6497_gb300 import build
    build.build()
    oracle.build()


def fill(plan, shapes, seed_offset=0):
    flat = plan.empty()
    fs = []
    for b, s in enumerate(shapes):
        f = wl.batch_instance(s, b + seed_offset).f.astype(np.float32)
        fs.append(f)
        plan.view(flat, b).copy_(torch.from_numpy(f))
    return flat, fs


def test_batch64_each_instance_matches_oracle():
    shapes = wl.batch_shapes(64)
    plan = Plan(dtype="f32", shapes=shapes)
    assert plan.launches_per_solve == 1
    flat, fs = fill(plan, shapes)
    u = plan.execute(flat)
    plan.status()
    worst = 0.0
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs[b].astype(np.float64))
        err, _ = check(plan.view(u, b).cpu().numpy(), ref, "f32", (b, s))
        worst = max(worst, err)
    total = sum(int(np.prod(s)) for s in shapes)
    print(f"batch of 64: {total} unknowns, worst rel-L2 {worst:.2e}")


def test_compile_time_and_run_time_plans_agree(monkeypatch):
    # every axis length of the batch draw: lines of 12…256 points run
    # compile-time plans by default, run-time plans with PSOLVE_BATCH_CT=0
    shapes = [(24, 32, 48), (64, 96, 128), (192, 256, 24), (48, 24, 192), (256, 64, 32)]
    plan = Plan(dtype="f32", shapes=shapes)
    flat, fs = fill(plan, shapes, seed_offset=50)
    u_ct = plan.execute(flat)
    plan.status()
    monkeypatch.setenv("PSOLVE_BATCH_CT", "0")
    plan_rt = Plan(dtype="f32", shapes=shapes)
    assert plan_rt.launches_per_solve == 1
    u_rt = plan_rt.execute(flat)
    plan_rt.status()
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs[b].astype(np.float64))
        a, r = plan.view(u_ct, b).cpu().numpy(), plan_rt.view(u_rt, b).cpu().numpy()
        check(a, ref, "f32", (s, "compile-time"))
        check(r, ref, "f32", (s, "run-time"))
        assert oracle.rel_l2(a, r) <= 1e-6, s


def test_graph_replay_new_data_and_new_buffers():
    shapes = [(24, 32, 48), (64, 24, 96), (32, 32, 32), (48, 128, 24)]
    plan = Plan(dtype="f32", shapes=shapes)
    flat1, fs1 = fill(plan, shapes)
    u1 = plan.execute(flat1)
    # same buffers, new contents
    flat2, fs2 = fill(plan, shapes, seed_offset=100)
    flat1.copy_(flat2)
    u1b = plan.execute(flat1, u1)
    # new buffers
    u2 = plan.execute(flat2.clone())
    plan.status()
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs2[b].astype(np.float64))
        check(plan.view(u1b, b).cpu().numpy(), ref, "f32")
        check(plan.view(u2, b).cpu().numpy(), ref, "f32")


def test_batched_matches_per_instance_launches(monkeypatch):
    shapes = wl.batch_shapes(6, seed=7)
    plan = Plan(dtype="f32", shapes=shapes)
    flat, _ = fill(plan, shapes)
    u_batched = plan.execute(flat)
    monkeypatch.setenv("PSOLVE_BATCHED", "0")
    plan2 = Plan(dtype="f32", shapes=shapes)
    assert plan2.launches_per_solve == 5 * len(shapes)
    u_loop = plan2.execute(flat)
    torch.cuda.synchronize()
    # same algorithm, different instruction schedules (compile-time plans and
    # the hardware reciprocal on the per-pass path): equal to FP32 rounding
    for b in range(len(shapes)):
        a, r = plan.view(u_batched, b), plan2.view(u_loop, b)
        assert float((a - r).norm() / r.norm()) <= 1e-6


def test_x_lines_too_long_for_a_batch_tile_run_per_pass():
    # 2048-point x lines need two 128-thread columns (256 threads) in the x
    # pass: the plan keeps one launch per pass and instance instead of failing
    shapes = [(2048, 4, 8), (8, 8, 8), (24, 48, 32)]
    plan = Plan(dtype="f32", shapes=shapes)
    assert plan.launches_per_solve == 5 * len(shapes)
    flat, fs = fill(plan, shapes, seed_offset=70)
    u = plan.execute(flat)
    plan.status()
    for b, s in enumerate(shapes):
        check(plan.view(u, b).cpu().numpy(), oracle.solve(fs[b].astype(np.float64)), "f32", s)


def test_bounded_wait_reports_timeout_and_context_survives():
    lib = _lib.load()
    shapes = [(8, 8, 8), (16, 8, 8)]
    plan = Plan(dtype="f32", shapes=shapes)
    flat, fs = fill(plan, shapes)
    # pass 1 of instance 0 now waits for a tile that does not exist
    assert lib.psolve_debug_set_wait(plan.handle, 50_000_000, 1) == 0
    plan.execute(flat)
    with pytest.raises(_lib.PsolveError) as ei:
        plan.status()
    assert ei.value.code == 5  # PSOLVE_ERR_TIMEOUT
    # restore the dependency: the same plan solves correctly again
    assert lib.psolve_debug_set_wait(plan.handle, 2_000_000_000, 0) == 0
    u = plan.execute(flat)
    plan.status()
    for b, s in enumerate(shapes):
        ref = oracle.solve(fs[b].astype(np.float64))
        check(plan.view(u, b).cpu().numpy(), ref, "f32")


def test_debug_wait_rejected_without_batched_launch():
    lib = _lib.load()
    plan = Plan((8, 8, 8), dtype="f32")
    assert lib.psolve_debug_set_wait(plan.handle, 1000, 1) == 1
